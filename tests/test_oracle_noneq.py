"""Pins of the oracle's non-equilibrium manifestations (Sec. II.E, Eqs.
M_absolute and D_absolute) by closed forms, the paper's identities and the
paper's sign criterion for shocks and rarefactions (Sec. III.C)."""
import math

import numpy as np
import pytest

from paper_1308_0653_gb300 import workloads as W

V = (1.5, 3.5, 7.5, 12.5)


def test_equilibrium_central_moments_are_the_maxwellians():
    """For f^eq: M*_2 = rho T I, M*_3 = 0, M*_{3,1} = 0 and
    M*_{4,2} = (1/2) rho (D + 2) T^2 I with D = 2 (continuous Maxwellian)."""
    rng = np.random.default_rng(7)
    for _ in range(30):
        th, rho, T = rng.uniform(0, 2 * math.pi), rng.uniform(0.3, 3), rng.uniform(0.5, 3)
        ur, uth = rng.uniform(-0.8, 0.8, 2) * math.sqrt(T)
        import oracle
        f = oracle.feq(th, rho, ur, uth, T, V)
        m = oracle.central_moments(th, f, ur, uth, V)
        s = rho * (1 + T) ** 2
        np.testing.assert_allclose(m[[0, 1, 2]], [rho * T, 0, rho * T], atol=1e-13 * s)
        np.testing.assert_allclose(m[3:9], 0.0, atol=1e-12 * s)
        np.testing.assert_allclose(m[[9, 10, 11]], [2 * rho * T * T, 0, 2 * rho * T * T], atol=1e-12 * s)


def test_paper_identities_of_the_contracted_third_moment(orc):
    """Sec. II.E: M*_{3,1,r} = (M*_{3,rrr} + M*_{3,r th th}) / 2 and
    M*_{3,1,th} = (M*_{3,rr th} + M*_{3,th th th}) / 2, for any g; and the
    same for Delta* (here on random non-equilibrium states)."""
    rng = np.random.default_rng(8)
    for _ in range(20):
        g = rng.uniform(-0.1, 0.3, 33)
        th, ur, uth = rng.uniform(0, 6.28), rng.uniform(-1, 1), rng.uniform(-1, 1)
        m = orc.central_moments(th, g, ur, uth, V)
        assert m[7] == pytest.approx(0.5 * (m[3] + m[5]), rel=1e-12, abs=1e-14)
        assert m[8] == pytest.approx(0.5 * (m[4] + m[6]), rel=1e-12, abs=1e-14)
    w = W.random_smooth(20, 16, seed=3, amp=0.2)
    p = orc.make_params(**{k: v for k, v in w.params.items() if k != "precision"})
    f, lam = orc.init(p, w.fields)
    f = f * (1 + 0.02 * rng.standard_normal(f.shape))
    d = orc.noneq(p, f)
    np.testing.assert_allclose(d[7], 0.5 * (d[3] + d[5]), atol=1e-12)
    np.testing.assert_allclose(d[8], 0.5 * (d[4] + d[6]), atol=1e-12)
    # T is f's own temperature, so the trace of Delta*_2 vanishes
    np.testing.assert_allclose(d[0] + d[2], 0.0, atol=1e-12)
    # f = f^eq carries no non-equilibrium
    f0, _ = orc.init(p, w.fields)
    np.testing.assert_allclose(orc.noneq(p, f0), 0.0, atol=1e-12)


def test_sign_of_delta2_rr_marks_shock_and_rarefaction(orc):
    """Sec. III.C: Delta*_{2,rr} is positive at a shock (compression) and
    negative at a rarefaction (expansion).  Planar shock tube at large radius:
    high pressure (rho 2, T 2) for r < 100.5 pushes a shock outwards and a
    rarefaction inwards."""
    nr, nth = 400, 8
    w = W.uniform_state(nr, nth, 1.0, 0.0, 0.0, 1.0, 0.0, r_in=100.0, r_out=101.0)
    r, th = W.grid(nr, nth, 100.0, 101.0)
    w.fields["rho"] = np.ascontiguousarray(np.where(r < 100.5, 2.0, 1.0))
    w.fields["T"] = np.ascontiguousarray(np.where(r < 100.5, 2.0, 1.0))
    dt = 0.4 * (1.0 / nr) / 12.5
    p = orc.make_params(**{**{k: v for k, v in w.params.items() if k != "precision"},
                           "dt": dt, "tau": 5e-4})
    f, lam = orc.init(p, w.fields)
    for _ in range(300):
        f, lam, _ = orc.step(p, f, lam)
    m = orc.macro(p, f, lam)
    d = orc.noneq(p, f)
    dudr = np.gradient(m["ur"][0], r[0])
    j_shock, j_rare = int(np.argmin(dudr)), int(np.argmax(dudr))
    assert r[0, j_shock] > 100.5 > r[0, j_rare]
    assert d[0, 0, j_shock] > 0 and d[2, 0, j_shock] < 0
    assert d[0, 0, j_rare] < 0 and d[2, 0, j_rare] > 0
    # far from both waves the gas is in equilibrium
    assert abs(d[0, 0, 5]) < 1e-3 * abs(d[0, 0, j_shock])
