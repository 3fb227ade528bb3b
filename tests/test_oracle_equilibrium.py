"""Pins of the oracle's velocity set, weights, equilibrium and chemical term
against what the mathematics fixes (Sec. II.A-II.B of the paper).

Each check compares with a closed form of the continuous Maxwellian (or an
exact identity of M), never with a retyped copy of the oracle's formula.
"""
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_numbers.json")))
V = GOLD["d2v33_speeds"]["value"]

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def test_velocity_set_geometry(orc):
    """Sec. II.B: 33 velocities, a rest particle and four rings of 8 at angles
    i pi/4, fixed in the Cartesian frame; polar components rotate with theta."""
    for theta in (0.0, 0.3, 2.0, 5.9):
        vr, vth = orc.velocities(theta, V)
        # Cartesian components are independent of theta.
        vx = vr * math.cos(theta) - vth * math.sin(theta)
        vy = vr * math.sin(theta) + vth * math.cos(theta)
        speeds = np.hypot(vx, vy)
        assert speeds[0] == 0.0
        for k in range(1, 5):
            ring = slice(1 + 8 * (k - 1), 1 + 8 * k)
            np.testing.assert_allclose(speeds[ring], V[k - 1], rtol=1e-15)
            # direction i sits at angle i pi/4 (index convention v = 1 + 8(k-1) + i)
            ang = np.arange(8) * math.pi / 4
            np.testing.assert_allclose(vx[ring], V[k - 1] * np.cos(ang), atol=1e-13)
            np.testing.assert_allclose(vy[ring], V[k - 1] * np.sin(ang), atol=1e-13)


@pytest.mark.parametrize("T", [0.3, 0.7, 1.0, 1.6, 2.6, 5.0])
def test_weights_reproduce_maxwellian_isotropic_moments(orc, T):
    """sum_{k,i} F_k v_k^{2n} = (2T)^n n! for n = 0..4 (2-D Maxwellian, unit
    density, zero velocity): the conditions the weights F_k are built from."""
    F = orc.weights(T, V)
    for n in range(5):
        s = F[0] * (1.0 if n == 0 else 0.0) + 8.0 * sum(F[k] * V[k - 1] ** (2 * n) for k in range(1, 5))
        assert s == pytest.approx((2 * T) ** n * math.factorial(n), rel=1e-13)


def test_printed_weight_sign_fails_the_moment_conditions():
    """Justifies the sign reading of F_k: with the printed '+1/4' on the last
    term the n = 1 moment (temperature) is wrong by a large factor."""
    T = 1.0
    x = [v * v for v in V]
    s = 0.0
    for k in range(4):
        a, b, c = x[(k + 1) % 4], x[(k + 2) % 4], x[(k + 3) % 4]
        den = x[k] * (x[k] - a) * (x[k] - b) * (x[k] - c)
        num = 48 * T ** 4 - 6 * (a + b + c) * T ** 3 + (a * b + b * c + c * a) * T ** 2 + 0.25 * a * b * c * T
        s += 8.0 * num / den * x[k]
    assert abs(s - 2 * T) > 0.1


def _rand_states(seed, n):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        theta = rng.uniform(0, 2 * math.pi)
        rho = rng.uniform(0.3, 3.0)
        T = rng.uniform(0.5, 3.0)
        umag = math.sqrt(T) * rng.uniform(0.0, 1.0)
        ang = rng.uniform(0, 2 * math.pi)
        yield theta, rho, umag * math.cos(ang), umag * math.sin(ang), T


def _maxwellian_moments(rho, u, T, D=2):
    I = np.eye(2)
    u2 = u @ u
    m2 = rho * (T * I + np.outer(u, u))
    m3 = rho * (np.einsum("a,b,c->abc", u, u, u)
                + T * (np.einsum("a,bc->abc", u, I) + np.einsum("b,ac->abc", u, I)
                       + np.einsum("c,ab->abc", u, I)))
    m31 = 0.5 * rho * u * (u2 + (D + 2) * T)
    m42 = 0.5 * rho * ((u2 + (D + 4) * T) * np.outer(u, u) + (u2 + (D + 2) * T) * T * I)
    return m2, m3, m31, m42


def test_feq_reproduces_maxwellian_moments(orc):
    """Eq. (feq): the discrete equilibrium has the continuous Maxwellian's
    density, momentum, temperature and its moments M2, M3, M3,1 and M4,2 (the
    set the Chapman-Enskog recovery of Sec. II.B rests on)."""
    for theta, rho, ur, uth, T in _rand_states(1, 40):
        f = orc.feq(theta, rho, ur, uth, T, V)
        vr, vth = orc.velocities(theta, V)
        Vm = np.stack([vr, vth])
        u = np.array([ur, uth])
        scale = rho * (1 + T) ** 3
        assert abs(f.sum() - rho) <= 1e-13 * rho
        np.testing.assert_allclose(Vm @ f, rho * u, atol=1e-13 * scale)
        c = Vm - u[:, None]
        assert 0.5 * np.einsum("ai,ai,i->", c, c, f) == pytest.approx(rho * T, rel=1e-12)
        m2, m3, m31, m42 = _maxwellian_moments(rho, u, T)
        np.testing.assert_allclose(np.einsum("ai,bi,i->ab", Vm, Vm, f), m2, atol=1e-12 * scale)
        np.testing.assert_allclose(np.einsum("ai,bi,ci,i->abc", Vm, Vm, Vm, f), m3, atol=1e-12 * scale)
        v2 = (Vm ** 2).sum(0)
        np.testing.assert_allclose(0.5 * np.einsum("i,ai,i->a", v2, Vm, f), m31, atol=1e-12 * scale)
        np.testing.assert_allclose(0.5 * np.einsum("i,ai,bi,i->ab", v2, Vm, Vm, f), m42,
                                   atol=1e-12 * scale)


def test_site_moments_invert_feq(orc):
    """Moments of f^eq(rho, u, T) give back (rho, u, T) (Sec. II.B definitions)."""
    for theta, rho, ur, uth, T in _rand_states(2, 40):
        f = orc.feq(theta, rho, ur, uth, T, V)
        r2, a, b, t2 = orc.site_moments(theta, f, V)
        assert r2 == pytest.approx(rho, rel=1e-14)
        assert a == pytest.approx(ur, abs=1e-13)
        assert b == pytest.approx(uth, abs=1e-13)
        assert t2 == pytest.approx(T, rel=1e-13)


def test_feq_is_frame_independent(orc):
    """f^eq of one Cartesian state seen from two site angles is the same
    function of the (Cartesian-fixed) velocity index."""
    rho, ux, uy, T = 1.3, 0.4, -0.25, 1.2
    ref = None
    for theta in (0.0, 0.7, 2.2, 4.0):
        ur = ux * math.cos(theta) + uy * math.sin(theta)
        uth = -ux * math.sin(theta) + uy * math.cos(theta)
        f = orc.feq(theta, rho, ur, uth, T, V)
        if ref is None:
            ref = f
        np.testing.assert_allclose(f, ref, rtol=1e-12, atol=1e-15)


def test_chemical_term_identities(orc):
    """Sec. II.A: sum M = 0, sum M v = 0 and (1/2) sum M v^2 = rho Q R, which
    the discrete M keeps because f^eq has the Maxwellian moments."""
    for theta, rho, ur, uth, T in _rand_states(3, 30):
        Q, R = 1.7, 0.37
        M = orc.chem(theta, rho, ur, uth, T, Q, R, V)
        vr, vth = orc.velocities(theta, V)
        scale = rho * Q * R * (1 + T) ** 2
        assert abs(M.sum()) <= 1e-13 * scale
        assert abs(M @ vr) <= 1e-12 * scale and abs(M @ vth) <= 1e-12 * scale
        assert 0.5 * M @ (vr ** 2 + vth ** 2) == pytest.approx(rho * Q * R, rel=1e-12)


def test_chemical_term_is_temperature_derivative(orc):
    """Eq. (M_chemical_4)-(M_continuous): M = (d f^eq / dT) dT/dt with
    dT/dt = (2Q/D) R.  For the discrete f^eq that is exact for the Maxwellian
    part; its zeroth to second moments match a finite difference of f^eq."""
    theta, rho, ur, uth, T = 0.4, 1.2, 0.3, -0.1, 1.5
    Q, R, D = 1.0, 0.8, 2
    h = 1e-5
    dfdT = (orc.feq(theta, rho, ur, uth, T + h, V) - orc.feq(theta, rho, ur, uth, T - h, V)) / (2 * h)
    M = orc.chem(theta, rho, ur, uth, T, Q, R, V)
    vr, vth = orc.velocities(theta, V)
    rate = 2 * Q / D * R
    for w in (np.ones(33), vr, vth, vr ** 2 + vth ** 2):
        assert M @ w == pytest.approx(dfdT @ w * rate, rel=1e-7, abs=1e-9)
