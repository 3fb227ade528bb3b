"""Pins of the oracle's reaction model (Sec. III.A): Cochran's rate, the
ignition gate, the exact one-step lambda update, and a homogeneous reactor
whose continuous solution has a closed form.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad, solve_ivp
from scipy.optimize import brentq

from paper_1308_0653_gb300 import workloads as W


def _params(orc, **kw):
    d = dict(nr=4, ntheta=8, r_in=1.0, r_out=2.0, dt=1e-3, tau=1e-3, omega1=2.0, omega2=3.0)
    d.update(kw)
    return orc.make_params(**d)


def test_cochran_rate_and_gate(orc):
    """R = w1 P^m (1 - lam) + w2 P^n lam (1 - lam) with P = rho T, zero unless
    T > T_th (strict)."""
    p = _params(orc, omega1=2.0, omega2=3.0, m=1.0, n=1.0, T_th=1.1)
    R, a, b = orc.rate(p, 1.5, 2.0, 0.25)
    P = 3.0
    assert a == pytest.approx(2.0 * P) and b == pytest.approx(3.0 * P)
    assert R == pytest.approx(2.0 * P * 0.75 + 3.0 * P * 0.25 * 0.75, rel=1e-15)
    assert orc.rate(p, 1.5, 1.1, 0.25) == (0.0, 0.0, 0.0)  # T == T_th: no reaction
    p2 = _params(orc, omega1=2.0, omega2=3.0, m=2.0, n=0.5)
    R2, a2, b2 = orc.rate(p2, 1.5, 2.0, 0.25)
    assert a2 == pytest.approx(2.0 * P ** 2) and b2 == pytest.approx(3.0 * P ** 0.5)


@pytest.mark.parametrize("lam0,a,b", [(0.0, 5.0, 0.0), (0.0, 1.0, 50.0), (0.3, 2.0, 7.0),
                                      (0.9, 0.5, 40.0), (0.999, 3.0, 3.0)])
def test_lambda_update_solves_the_rate_ode(orc, lam0, a, b):
    """Eq. (Eqlambda), reaction part: with a, b frozen the update equals the
    solution of d lam/dt = (1 - lam)(a + b lam) at t = dt (checked against a
    high-accuracy numerical integration), for small and large a dt, b dt."""
    for dt in (1e-4, 1e-2, 0.3):
        sol = solve_ivp(lambda t, y: (1 - y) * (a + b * y), (0, dt), [lam0], rtol=1e-12,
                        atol=1e-14, method="DOP853")
        assert orc.lambda_react(lam0, a, b, dt) == pytest.approx(sol.y[0, -1], abs=2e-11)


def test_lambda_update_is_a_semigroup(orc):
    """Exact flow: two steps of dt equal one step of 2 dt."""
    for lam0, a, b in [(0.0, 3.0, 10.0), (0.4, 1.0, 1.0), (0.8, 0.0, 6.0)]:
        one = orc.lambda_react(lam0, a, b, 0.02)
        two = orc.lambda_react(orc.lambda_react(lam0, a, b, 0.01), a, b, 0.01)
        assert one == pytest.approx(two, abs=1e-15)


def test_lambda_update_limits(orc):
    """No reaction (a = b = 0) leaves lam; lam = 1 is a fixed point; from
    lam = 0 with b = 0 the result is 1 - exp(-a dt) (not the printed form's
    tanh(a dt / 2), which starts at half the rate)."""
    assert orc.lambda_react(0.37, 0.0, 0.0, 0.1) == 0.37
    assert orc.lambda_react(1.0, 2.0, 5.0, 0.1) == pytest.approx(1.0, abs=1e-15)
    a, dt = 4.0, 0.05
    assert orc.lambda_react(0.0, a, 0.0, dt) == pytest.approx(1 - math.exp(-a * dt), rel=1e-14)
    assert abs(orc.lambda_react(0.0, a, 0.0, dt) - math.tanh(a * dt / 2)) > 0.03


def _homogeneous_run(orc, dt, t_end, mode, rho=1.0, T0=1.5, w1=2.0, w2=2.0, Q=1.0):
    """Uniform reactant at rest: no gradients, so only collision and reaction act."""
    w = W.uniform_state(4, 8, rho, 0.0, 0.0, T0, 0.0, r_in=1.0, r_out=2.0)
    p = orc.make_params(**{k: v for k, v in w.params.items() if k != "precision"})
    p.dt, p.tau, p.omega1, p.omega2, p.Q, p.reaction_energy = dt, 1e-3, w1, w2, Q, mode
    f, lam = orc.init(p, w.fields)
    n = int(round(t_end / dt))
    for _ in range(n):
        f, lam, _c = orc.step(p, f, lam)
    m = orc.macro(p, f, lam)
    return m


def _exact_lambda(t, rho=1.0, T0=1.5, w1=2.0, w2=2.0, Q=1.0):
    """Continuous homogeneous reactor with D = 2: dT/dt = (2Q/D) R = Q R and
    d lam/dt = R, so T = alpha + Q lam (alpha = T0) and
    d lam/dt = rho (alpha + Q lam)(1 - lam)(w1 + w2 lam); t(lam) by quadrature."""
    def g(l):
        return rho * (T0 + Q * l) * (1 - l) * (w1 + w2 * l)
    return brentq(lambda lam: quad(lambda l: 1 / g(l), 0, lam, epsabs=1e-14, epsrel=1e-13)[0] - t,
                  0.0, 0.99, xtol=1e-15)


def test_homogeneous_reactor_converges_first_order(orc):
    """The coupled update (M heating + exact lambda step) converges to the
    continuous reactor at first order in dt, and T - Q lam stays constant to
    O(dt) (explicit R) or to round-off (R taken as the step's increment)."""
    t_end = 0.2
    lam_ex = _exact_lambda(t_end)
    errs = []
    for dt in (2e-3, 1e-3, 5e-4):
        m = _homogeneous_run(orc, dt, t_end, mode=0)
        lam = m["lam"].mean()
        # uniform state stays uniform
        assert np.ptp(m["lam"]) < 1e-13 and np.ptp(m["T"]) < 1e-13
        errs.append(abs(lam - lam_ex))
    assert errs[-1] < 2e-3
    for e1, e2 in zip(errs, errs[1:]):
        assert 1.7 < e1 / e2 < 2.3, errs
    m = _homogeneous_run(orc, 1e-3, t_end, mode=1)
    inv = m["T"] - 1.0 * m["lam"]
    assert np.abs(inv - 1.5).max() < 1e-12
    assert abs(m["lam"].mean() - lam_ex) < 2e-3
    m0 = _homogeneous_run(orc, 1e-3, t_end, mode=0)
    drift = np.abs(m0["T"] - m0["lam"] - 1.5).max()
    assert 1e-6 < drift < 1e-2
