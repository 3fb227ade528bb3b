"""Pins of the ZND structure solver (oracle/znd.py) against textbook results
it does not use: the CJ closed form, the sonic condition at the CJ point, the
normal-shock jump relations, and the exact reaction-zone length of a wave
without heat release."""
import math

import numpy as np
import pytest

from oracle import znd
from test_oracle_cj import GOLD, cj_state


def test_cj_speed_by_bisection_equals_the_closed_form_and_the_papers_number():
    D = znd.cj_speed()
    assert D == pytest.approx(cj_state()[0], rel=1e-12)
    assert D == pytest.approx(GOLD["cj_speed"]["value"], abs=1e-5)


def test_cj_point_is_sonic_and_is_the_papers_burnt_state():
    """At lambda = 1 the burnt gas leaves the front at its own sound speed
    sqrt(gamma P / rho), and the state is the paper's initial burnt state."""
    D = znd.cj_speed()
    rho, P, T, u = znd.state(1.0, D)
    w = D - u
    assert w == pytest.approx(math.sqrt(2.0 * P / rho), rel=1e-6)
    g = GOLD["cj_initial_burnt_state"]
    assert rho == pytest.approx(g["rho"], abs=1e-5)
    assert T == pytest.approx(g["T"], abs=1e-5)
    assert u == pytest.approx(g["u_r"], abs=1e-5)


@pytest.mark.parametrize("D", [2.0, 3.0, 3.09557, 5.0])
def test_von_neumann_state_is_the_normal_shock_jump(D):
    """lambda = 0: the ideal-gas normal shock of Mach M = D / c0 (gamma = 2)."""
    g, c0 = 2.0, math.sqrt(2.0)
    M2 = (D / c0) ** 2
    rho, P, T, u = znd.state(0.0, D, Q=0.0)
    assert rho == pytest.approx((g + 1) * M2 / ((g - 1) * M2 + 2), rel=1e-12)
    assert P == pytest.approx(1.0 + 2 * g / (g + 1) * (M2 - 1), rel=1e-12)
    assert u == pytest.approx(D * (1 - 1 / rho), rel=1e-12)


def test_fluxes_are_constant_through_the_reaction_zone():
    z = znd.profile(npts=2001)
    D = z["D"]
    w = D - z["u"]
    np.testing.assert_allclose(z["rho"] * w, D, rtol=1e-12)
    np.testing.assert_allclose(z["P"] + z["rho"] * w ** 2, 1.0 + D * D, rtol=1e-12)
    np.testing.assert_allclose(2 * z["T"] + w ** 2 / 2 - z["lam"], 2.0 + D * D / 2, rtol=1e-12)
    assert np.all(np.diff(z["x"]) > 0)
    assert np.all(np.diff(z["P"]) < 0)  # pressure falls from the spike to CJ


def test_zone_length_without_heat_release_is_logarithmic():
    """Q = 0, omega2 = 0: the shocked state is uniform, R = omega1 P1^m (1 - lam),
    so x(lam) = -w1 ln(1 - lam) / (omega1 P1^m) exactly."""
    D, om1, m = 3.0, 7.0, 1.0
    z = znd.profile(D=D, Q=0.0, omega1=om1, omega2=0.0, m=m, n=1.0, lam_max=1 - 1e-5)
    rho1, P1, _, u1 = znd.state(0.0, D, Q=0.0)
    exact = -(D - u1) * np.log1p(-z["lam"]) / (om1 * P1 ** m)
    np.testing.assert_allclose(z["x"][1:], exact[1:], rtol=1e-6)


def test_zone_length_with_both_rate_terms_has_its_closed_form():
    """Q = 0 keeps the shocked state uniform, so with a = omega1 P1^m and
    b = omega2 P1^n the rate is (1 - lam)(a + b lam) and, by partial
    fractions, x(lam) = w1 / (a + b) ln[(a + b lam) / (a (1 - lam))].  The
    exponents differ (m = 1, n = 2) and P1 = 5.67 is far from 1, so each
    term must carry its own exponent and the second its factor lam.  (b / a
    is kept near 1.6: the integral is a midpoint rule, and a steeper rate
    near lam = 0 would show its second-order error above 1e-6.)"""
    D, om1, om2, m, n = 3.0, 7.0, 2.0, 1.0, 2.0
    z = znd.profile(D=D, Q=0.0, omega1=om1, omega2=om2, m=m, n=n, lam_max=1 - 1e-5)
    rho1, P1, _, u1 = znd.state(0.0, D, Q=0.0)
    assert P1 == pytest.approx(1.0 + 4.0 / 3.0 * (D * D / 2.0 - 1.0), rel=1e-12)
    a, b = om1 * P1 ** m, om2 * P1 ** n
    lam = z["lam"][1:]
    exact = (D - u1) / (a + b) * np.log((a + b * lam) / (a * (1.0 - lam)))
    np.testing.assert_allclose(z["x"][1:], exact, rtol=1e-6)


def test_below_cj_speed_there_is_no_steady_wave():
    with pytest.raises(ValueError):
        znd.state(1.0, 0.99 * znd.cj_speed())
