"""Steady ZND detonation structure of the model gas (test infrastructure only).

Only tests/ may import this module.  It shares nothing with the CUDA path.

The discrete Boltzmann model of Sec. II describes an ideal gas with D = 2
translational degrees of freedom: internal energy T per unit mass, P = rho T,
so gamma = (D + 2) / D = 2.  The chemical term of Sec. II.C releases Q per
unit mass of reactant burnt, and lambda (reacted fraction) obeys Cochran's
rate, Sec. III.A: d lambda / dt = (1 - lambda)(omega1 P^m + omega2 P^n lambda)
while T > T_th, zero otherwise.

A ZND wave is a shock of speed D into the fresh gas followed by a steady,
inviscid reaction zone.  In the frame moving with the shock (w = D - u, the
gas speed relative to the front) the flux of mass, momentum and total
enthalpy is the same at every point of the zone:

    rho w = rho0 D =: j
    P + rho w^2 = P0 + rho0 D^2
    gamma/(gamma-1) P/rho + w^2/2 - lambda Q = gamma/(gamma-1) P0/rho0 + D^2/2

For a given lambda these fix the state (the Rayleigh line meets the partial
Hugoniot curve of heat release lambda Q): with the specific volume
v = 1/rho and P = P0 + j^2 (v0 - v), the energy balance is a quadratic in v,
whose smaller root is the shocked (ZND) branch.  The position behind the
shock follows from the rate, w d lambda / dx = R, so x(lambda) is the
integral of w / R.  The Chapman-Jouguet speed is the D at which the two roots
meet at lambda = 1 (the burnt gas leaves the front at its sound speed).
"""
import math

import numpy as np


def _hugoniot(lam, D, Q, gamma, rho0, P0):
    """State on the ZND branch at reacted fraction lam: (rho, P, T, u, w, disc).
    disc < 0 means no steady state exists at this speed (D below CJ)."""
    j = rho0 * D
    v0 = 1.0 / rho0
    g = gamma / (gamma - 1.0)
    # g (P0 + j^2 (v0 - v)) v + j^2 v^2 / 2 = g P0 v0 + j^2 v0^2 / 2 + lam Q
    a = (g - 0.5) * j * j
    b = g * (P0 + j * j * v0)
    c = g * P0 * v0 + 0.5 * j * j * v0 * v0 + lam * Q
    disc = b * b - 4.0 * a * c
    v = (b - math.sqrt(max(disc, 0.0))) / (2.0 * a)
    P = P0 + j * j * (v0 - v)
    rho = 1.0 / v
    w = j * v
    return rho, P, P / rho, D - w, w, disc


def cj_speed(Q=1.0, gamma=2.0, rho0=1.0, P0=1.0, tol=1e-14):
    """The Chapman-Jouguet speed: the smallest D whose Hugoniot at lam = 1 has
    a real state, found by bisection on the discriminant (no closed form used)."""
    c0 = math.sqrt(gamma * P0 / rho0)
    lo, hi = c0, c0 + 10.0 * math.sqrt(Q) + 10.0
    assert _hugoniot(1.0, hi, Q, gamma, rho0, P0)[5] > 0
    while hi - lo > tol * hi:
        mid = 0.5 * (lo + hi)
        if _hugoniot(1.0, mid, Q, gamma, rho0, P0)[5] >= 0:
            hi = mid
        else:
            lo = mid
    return hi


def state(lam, D, Q=1.0, gamma=2.0, rho0=1.0, P0=1.0):
    """Lab-frame state (rho, P, T, u) at reacted fraction lam of a steady wave
    of speed D; lam = 0 is the von Neumann state just behind the shock."""
    rho, P, T, u, _, disc = _hugoniot(lam, D, Q, gamma, rho0, P0)
    if disc < -1e-9 * D ** 4:
        raise ValueError("no steady state: D is below the Chapman-Jouguet speed")
    return rho, P, T, u


def profile(D=None, Q=1.0, omega1=10.0, omega2=1000.0, m=1.0, n=1.0, T_th=1.1, gamma=2.0,
            rho0=1.0, P0=1.0, lam_max=1.0 - 1e-6, npts=20001):
    """ZND profile behind the shock: arrays x (distance behind the shock),
    lam, rho, P, T, u (lab frame), for lam in [0, lam_max].  D defaults to
    the CJ speed.  The integral of w / R is taken by the midpoint rule on a
    lambda grid clustered towards lam_max (R ~ (1 - lam) there)."""
    if D is None:
        D = cj_speed(Q, gamma, rho0, P0)
    # lambda grid: uniform in -log(1 - lam) so the logarithmic tail is resolved
    s = np.linspace(0.0, -math.log(1.0 - lam_max), npts)
    lam = 1.0 - np.exp(-s)
    x = np.zeros(npts)
    for i in range(1, npts):
        lm = 0.5 * (lam[i - 1] + lam[i])
        _, P, T, _, w, _ = _hugoniot(lm, D, Q, gamma, rho0, P0)
        if not T > T_th:
            raise ValueError("the shocked gas is below the ignition temperature")
        R = (1.0 - lm) * (omega1 * P ** m + omega2 * P ** n * lm)
        x[i] = x[i - 1] + w / R * (lam[i] - lam[i - 1])
    st = np.array([state(l, D, Q, gamma, rho0, P0) if l < 1.0 else state(1.0, D, Q, gamma, rho0, P0)
                   for l in lam])
    return dict(x=x, lam=lam, rho=st[:, 0], P=st[:, 1], T=st[:, 2], u=st[:, 3], D=D)
