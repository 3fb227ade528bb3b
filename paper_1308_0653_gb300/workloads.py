"""Seeded synthetic workloads: parameters and macroscopic initial fields.

This module is the one piece shared by the CUDA path and the CPU oracle.  It
holds none of the method's arithmetic (no equilibrium, no moments, no update):
it only lays out initial (rho, u_r, u_theta, T, lambda) fields on the polar
grid and draws seeded random numbers with a counter-based generator
(SplitMix64, Steele, Lea and Flood, OOPSLA 2014), so both sides see the same
inputs.

Grid convention: r_j = r_in + (j + 1/2) dr with dr = (r_out - r_in)/nr and
theta_m = m * 2 pi / ntheta; fields are float64 arrays of shape (ntheta, nr).

Workload shapes follow the paper's runs: a hot reacted ring igniting premixed
reactant (explosion, Sec. III.D), a shocked outer ring driven inwards
(implosion, Sec. III.C), and the planar Chapman-Jouguet detonation of the
validation run (Sec. III.B), all with the paper's D2V33 speeds, Cochran
exponents m = n = 1, ignition temperature 1.1 and heat release Q = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15

PAPER_SPEEDS = (1.5, 3.5, 7.5, 12.5)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on uint64 arrays (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, stream: int, n: int) -> np.ndarray:
    """n 64-bit outputs of SplitMix64 for counter i = 0..n-1 of (seed, stream)."""
    key = int(_mix64(np.array([(seed * _GOLDEN + stream + 1) & _MASK], dtype=np.uint64))[0])
    ctr = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = np.uint64(key) + ctr * np.uint64(_GOLDEN)
    return _mix64(x)


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles uniform in [0, 1) (top 53 bits of SplitMix64)."""
    return (splitmix64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_at(seed: int, stream: int, i: int) -> float:
    """The i-th value (from 0) of uniform(seed, stream, .), computed alone."""
    key = int(_mix64(np.array([(seed * _GOLDEN + stream + 1) & _MASK], dtype=np.uint64))[0])
    x = np.array([(key + (i + 1) * _GOLDEN) & _MASK], dtype=np.uint64)
    return float((_mix64(x) >> np.uint64(11)).astype(np.float64)[0] * (2.0 ** -53))


@dataclass
class Workload:
    """Parameters (paper names) + initial fields + number of time steps."""
    name: str
    params: dict
    fields: dict
    nsteps: int
    meta: dict = field(default_factory=dict)

    @property
    def sites(self) -> int:
        return int(self.params["nr"]) * int(self.params["ntheta"])


def grid(nr: int, ntheta: int, r_in: float, r_out: float, sector: int = 0):
    """(r, theta) broadcast grids of shape (ntheta, nr) (theta span 2 pi, or
    pi/4 for a sector)."""
    dr = (r_out - r_in) / nr
    r = r_in + (np.arange(nr) + 0.5) * dr
    th = np.arange(ntheta) * ((math.pi / 4 if sector else 2.0 * math.pi) / ntheta)
    return np.broadcast_to(r[None, :], (ntheta, nr)), np.broadcast_to(th[:, None], (ntheta, nr))


def base_params(**kw) -> dict:
    p = dict(r_in=0.05, r_out=1.05, dt=1e-5, tau=1e-3, Q=1.0, omega1=0.0, omega2=0.0,
             m=1.0, n=1.0, T_th=1.1, v=PAPER_SPEEDS, reaction_energy=0, precision="fp32")
    p.update(kw)
    return p


def _two_state(nr, ntheta, r_in, r_out, inside, state_in, state_out, sector=0):
    r, th = grid(nr, ntheta, r_in, r_out, sector)
    mask = inside(r, th)
    out = {}
    for i, name in enumerate(("rho", "ur", "uth", "T", "lam")):
        out[name] = np.where(mask, float(state_in[i]), float(state_out[i])).astype(np.float64)
    return out


def explosion64(precision: str = "fp64") -> Workload:
    """Non-reactive cylindrical explosion on a 64 x 64 annulus, 200 steps."""
    p = base_params(nr=64, ntheta=64, dt=1e-5, tau=1e-3, omega1=0.0, omega2=0.0,
                    precision=precision)
    f = _two_state(64, 64, p["r_in"], p["r_out"], lambda r, th: r < 0.3,
                   (2.0, 0.0, 0.0, 2.0, 0.0), (1.0, 0.0, 0.0, 1.0, 0.0))
    return Workload("explosion64", p, f, 200)


def explosion(nr: int = 512, ntheta: int = 512, nsteps: int = 5000, seed: int = 0,
              precision: str = "fp32", omega1: float = 2.0, omega2: float = 2.0,
              r_hot: float = 0.2, dt: float = 1e-5) -> Workload:
    """Reactive cylindrical explosion: a hot reacted ring (rho 1.4, T 1.6,
    lambda 1) for r < r_hot igniting premixed reactant (rho 1, T 1, lambda 0),
    with 1% white noise on rho drawn from (seed, stream 1)."""
    p = base_params(nr=nr, ntheta=ntheta, dt=dt, tau=1e-3, omega1=omega1, omega2=omega2,
                    precision=precision)
    f = _two_state(nr, ntheta, p["r_in"], p["r_out"], lambda r, th: r < r_hot,
                   (1.4, 0.0, 0.0, 1.6, 1.0), (1.0, 0.0, 0.0, 1.0, 0.0))
    xi = 2.0 * uniform(seed, 1, nr * ntheta).reshape(ntheta, nr) - 1.0
    f["rho"] = f["rho"] * (1.0 + 0.01 * xi)
    return Workload(f"explosion{nr}x{ntheta}", p, f, nsteps, dict(seed=seed))


def implosion(nr: int = 2048, ntheta: int = 2048, nsteps: int = 20000, seed: int = 0,
              precision: str = "fp32", omega1: float = 2.0, omega2: float = 2.0,
              dt: float = 5e-6, r_shock: float = 0.9) -> Workload:
    """Reactive implosion: for r > r_s(theta) a shocked reacted ring (rho 1.4,
    T 1.6, u_r -0.5, lambda 1) drives inwards into reactant (rho 1, T 1,
    lambda 0).  r_s(theta) = r_shock [1 + 0.005 sum_{q=4}^{16} a_q cos(q theta +
    phi_q) / sum a_q] with a_q ~ U(0,1) (stream 2), phi_q ~ U(0, 2 pi) (stream 3)."""
    p = base_params(nr=nr, ntheta=ntheta, dt=dt, tau=1e-3, omega1=omega1, omega2=omega2,
                    precision=precision)
    modes = np.arange(4, 17)
    amp = uniform(seed, 2, modes.size)
    phase = 2.0 * math.pi * uniform(seed, 3, modes.size)

    def outside(r, th):
        # r_s depends on theta alone: one value per row, broadcast over the row's sites
        t = th[:, :1]
        pert = (amp[None, None, :] * np.cos(modes[None, None, :] * t[..., None]
                                            + phase[None, None, :])).sum(-1) / amp.sum()
        return r > r_shock * (1.0 + 0.005 * pert)

    f = _two_state(nr, ntheta, p["r_in"], p["r_out"], outside,
                   (1.4, -0.5, 0.0, 1.6, 1.0), (1.0, 0.0, 0.0, 1.0, 0.0))
    return Workload(f"implosion{nr}x{ntheta}", p, f, nsteps, dict(seed=seed))


def planar_cj(nr: int = 20000, ntheta: int = 8, dt: float = 2.5e-7, t_end: float = 0.025,
              precision: str = "fp64", sector: int = 0) -> Workload:
    """Steady planar detonation of the validation run (Sec. III.B): annulus
    r in [1000, 1000.1]; Chapman-Jouguet burnt state (1.35826, 2.59709, 0.81650,
    0, 1) for r <= 1000.01, unburnt (1, 1, 0, 0, 0) outside; tau 2e-4,
    omega1 10, omega2 1000.  ntheta = 8 with axisymmetric data on a full 2 pi
    grid reproduces the paper's one-cell pi/4 sector (sector = 1, ntheta = 1)."""
    p = base_params(nr=nr, ntheta=ntheta, r_in=1000.0, r_out=1000.1, dt=dt, tau=2e-4,
                    omega1=10.0, omega2=1000.0, precision=precision, sector=sector)
    f = _two_state(nr, ntheta, 1000.0, 1000.1, lambda r, th: r <= 1000.01,
                   (1.35826, 0.81650, 0.0, 2.59709, 1.0), (1.0, 0.0, 0.0, 1.0, 0.0), sector)
    return Workload(f"planar_cj{nr}", p, f, int(round(t_end / dt)))


def uniform_state(nr: int, ntheta: int, rho: float, ux: float, uy: float, T: float,
                  lam: float = 0.0, **kw) -> Workload:
    """A spatially uniform state with Cartesian velocity (ux, uy): its polar
    components vary with theta as u_r = ux cos + uy sin, u_th = -ux sin + uy cos."""
    p = base_params(nr=nr, ntheta=ntheta, **kw)
    r, th = grid(nr, ntheta, p["r_in"], p["r_out"], p.get("sector", 0))
    f = dict(rho=np.full((ntheta, nr), float(rho)),
             ur=ux * np.cos(th) + uy * np.sin(th),
             uth=-ux * np.sin(th) + uy * np.cos(th),
             T=np.full((ntheta, nr), float(T)),
             lam=np.full((ntheta, nr), float(lam)))
    f = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in f.items()}
    return Workload(f"uniform{nr}x{ntheta}", p, f, 0)


def random_smooth(nr: int, ntheta: int, seed: int = 0, amp: float = 0.1, **kw) -> Workload:
    """Smooth random fields (a few seeded Fourier modes in r and theta) around
    rho = 1, T = 1.3, u = 0, lambda = 0.3, for parity tests of every term."""
    p = base_params(nr=nr, ntheta=ntheta, **kw)
    r, th = grid(nr, ntheta, p["r_in"], p["r_out"], p.get("sector", 0))
    x = (r - p["r_in"]) / (p["r_out"] - p["r_in"])
    out = {}
    base = dict(rho=1.0, ur=0.0, uth=0.0, T=1.3, lam=0.3)
    for s, name in enumerate(("rho", "ur", "uth", "T", "lam")):
        c = uniform(seed, 10 + s, 8)
        val = np.full((ntheta, nr), base[name])
        for q in range(2):
            a, b, ph1, ph2 = c[4 * q:4 * q + 4]
            val = val + amp * (a - 0.5) * np.cos(2 * math.pi * (q + 1) * x + 6.28 * ph1) \
                            * np.cos((q + 1) * th + 6.28 * ph2) + amp * (b - 0.5) * np.sin((q + 2) * th)
        out[name] = np.ascontiguousarray(val, dtype=np.float64)
    out["lam"] = np.clip(out["lam"], 0.0, 1.0)
    return Workload(f"smooth{nr}x{ntheta}", p, out, 0, dict(seed=seed))


def batch(n_instances: int = 64, seed: int = 0, nsteps: int = 5000, nmin: int = 128,
          nmax: int = 1024, precision: str = "fp32", align: int = 1) -> list:
    """Batched sweep: square N x N grids with N uniform in [nmin, nmax]
    (stream 20, rounded down to a multiple of `align`), driver pressure ratio
    s ~ logU[1.2, 3] (stream 21, rho_hot = T_hot = sqrt(s)), omega1 ~
    logU[0.5, 8] (stream 22), explosion and implosion alternating, and
    dt = 0.4 min(dr, r_in dtheta) / 12.5."""
    un = uniform(seed, 20, n_instances)
    us = uniform(seed, 21, n_instances)
    uw = uniform(seed, 22, n_instances)
    out = []
    for i in range(n_instances):
        N = nmin + int(un[i] * (nmax - nmin + 1))
        N = max(nmin, (N // align) * align)
        s = 1.2 * (3.0 / 1.2) ** us[i]
        w1 = 0.5 * (8.0 / 0.5) ** uw[i]
        hot = math.sqrt(s)
        dr = 1.0 / N
        dt = 0.4 * min(dr, 0.05 * 2 * math.pi / N) / 12.5
        if i % 2 == 0:
            p = base_params(nr=N, ntheta=N, dt=dt, tau=1e-3, omega1=w1, omega2=2.0,
                            precision=precision)
            f = _two_state(N, N, p["r_in"], p["r_out"], lambda r, th: r < 0.2,
                           (hot, 0.0, 0.0, hot, 1.0), (1.0, 0.0, 0.0, 1.0, 0.0))
            name = f"b{i}_explosion{N}"
        else:
            p = base_params(nr=N, ntheta=N, dt=dt, tau=1e-3, omega1=w1, omega2=2.0,
                            precision=precision)
            f = _two_state(N, N, p["r_in"], p["r_out"], lambda r, th: r > 0.9,
                           (hot, -0.5, 0.0, hot, 1.0), (1.0, 0.0, 0.0, 1.0, 0.0))
            name = f"b{i}_implosion{N}"
        out.append(Workload(name, p, f, nsteps, dict(seed=seed, index=i, ratio=s)))
    return out


def arrivals(rate_hz: float, duration_s: float, seed: int = 0):
    """Poisson arrival times (exponential gaps, stream 30) within duration_s."""
    n = max(16, int(rate_hz * duration_s * 1.5) + 16)
    while True:
        gaps = -np.log1p(-uniform(seed, 30, n)) / rate_hz
        t = np.cumsum(gaps)
        if t[-1] >= duration_s:
            return [float(x) for x in t[t < duration_s]]
        n *= 2


def serving_shape(k: int, seed: int = 0, nmin: int = 128, nmax: int = 2048,
                  smin: int = 1000, smax: int = 20000, align: int = 32):
    """(N, steps, explosion?, omega1) of request k of the serving stream, without
    its fields: side N ~ logU[nmin, nmax] (stream 31, multiple of `align`),
    steps ~ logU[smin, smax] (stream 32), explosion or implosion with equal
    odds (stream 33), omega1 in {1, 2, 4} (stream 34)."""
    u = [uniform_at(seed, 31 + s, k) for s in range(4)]
    N = int(nmin * (nmax / nmin) ** u[0])
    N = max(align, (N // align) * align)
    steps = int(smin * (smax / smin) ** u[1])
    w1 = (1.0, 2.0, 4.0)[min(2, int(u[3] * 3))]
    return N, steps, u[2] < 0.5, w1


def serving_request(k: int, seed: int = 0, nmin: int = 128, nmax: int = 2048,
                    smin: int = 1000, smax: int = 20000, align: int = 32) -> Workload:
    """Request k of the serving stream (shape as serving_shape)."""
    N, steps, is_explosion, w1 = serving_shape(k, seed, nmin, nmax, smin, smax, align)
    dt = 0.4 * min(1.0 / N, 0.05 * 2 * math.pi / N) / 12.5
    if is_explosion:
        w = explosion(N, N, steps, seed=seed + k, omega1=w1, dt=dt)
    else:
        w = implosion(N, N, steps, seed=seed + k, omega1=w1, dt=dt)
    w.name = f"req{k}_{w.name}"
    return w


def paper_explosion(R1: float, R: float, nr: int, dt: float = 1.25e-6, nsteps: int = 0,
                    precision: str = "fp32") -> Workload:
    """The paper's explosion runs (Sec. III.D): a disc of radius R in one pi/4
    sector cell (ntheta = 1) with the centre rule; reacted driver (rho, T,
    u_r, u_theta, lambda) = (1.5, 1.55556, 0.666667, 0, 1) for r <= R1 into
    (1, 1, 0, 0, 0); tau 2e-4, omega1 1, omega2 50.  The paper's cases are
    (R1, R, nr) = (0.015, 0.3, 6000), (0.023, 0.75, 15000), (0.05, 1.2, 24000)
    with dt 2.5e-6; dt defaults to half of that (Courant sum <= 1 at the
    innermost cell)."""
    p = base_params(nr=nr, ntheta=1, r_in=0.0, r_out=R, dt=dt, tau=2e-4, omega1=1.0,
                    omega2=50.0, precision=precision, sector=1, r_bc_inner="centre")
    f = _two_state(nr, 1, 0.0, R, lambda r, th: r <= R1,
                   (1.5, 0.666667, 0.0, 1.55556, 1.0), (1.0, 0.0, 0.0, 1.0, 0.0))
    return Workload(f"paper_explosion_R1_{R1}", p, f, nsteps, dict(R1=R1, R=R))


def paper_implosion(nr: int = 2000, dt: float = 1.25e-6, nsteps: int = 0,
                    precision: str = "fp32") -> Workload:
    """The paper's implosion run (Sec. III.C): disc of radius 0.1, one pi/4
    sector cell, centre rule; shocked reacted ring (1.5, 1.55556, -0.666667,
    0, 1) for 0.098 < r <= 0.1 driving into (1, 1, 0, 0, 0); tau 2e-4,
    omega1 1, omega2 50; the paper's nr = 2000 with dt 2.5e-6 (default here
    half of that)."""
    p = base_params(nr=nr, ntheta=1, r_in=0.0, r_out=0.1, dt=dt, tau=2e-4, omega1=1.0,
                    omega2=50.0, precision=precision, sector=1, r_bc_inner="centre")
    f = _two_state(nr, 1, 0.0, 0.1, lambda r, th: r > 0.098,
                   (1.5, -0.666667, 0.0, 1.55556, 1.0), (1.0, 0.0, 0.0, 1.0, 0.0))
    return Workload("paper_implosion", p, f, nsteps)
