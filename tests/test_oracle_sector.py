"""Pins of the oracle's sector and disc-centre geometry (Sec. II.D, Fig. 1).

A pi/4 sector with the rotated periodic wrap and a full 2 pi grid carrying
8-fold symmetric data are the same physical problem; so are the paper's
centre rule in a sector (i -> i+4 at the same theta) and the mirror point
across the centre on a full grid.  Equal results pin both readings."""
import math

import numpy as np
import pytest

from paper_1308_0653_gb300 import workloads as W


def _sector_fields(nr, s, r_in, r_out, seed):
    """Smooth random fields on a sector grid of s rows (span pi/4)."""
    rng = np.random.default_rng(seed)
    dr = (r_out - r_in) / nr
    r = r_in + (np.arange(nr) + 0.5) * dr
    th = (np.arange(s) + 0.0) * (math.pi / 4 / s)
    R, TH = np.meshgrid(r, th)
    x = (R - r_in) / (r_out - r_in)
    f = {}
    base = dict(rho=1.0, ur=0.0, uth=0.0, T=1.3, lam=0.3)
    for k, name in enumerate(("rho", "ur", "uth", "T", "lam")):
        c = rng.uniform(-1, 1, 4)
        val = base[name] + 0.15 * (c[0] * np.cos(2 * math.pi * x + c[1]) * np.cos(8 * TH + c[2])
                                   + c[3] * np.sin(3 * math.pi * x))
        f[name] = np.ascontiguousarray(val)
    f["lam"] = np.clip(f["lam"], 0, 1)
    f["T"] = np.abs(f["T"]) + 0.5
    f["rho"] = np.abs(f["rho"]) + 0.3
    return f


def _run(orc, fields, nr, nth, r_in, r_out, sector, centre, nsteps, dt):
    p = orc.make_params(nr=nr, ntheta=nth, r_in=r_in, r_out=r_out, dt=dt, tau=5e-4,
                        omega1=3.0, omega2=4.0, sector=sector, r_bc_inner=centre)
    f, lam = orc.init(p, fields)
    for _ in range(nsteps):
        f, lam, _ = orc.step(p, f, lam)
    return orc.macro(p, f, lam), f


@pytest.mark.parametrize("centre,r_in", [(0, 0.4), (1, 0.0)])
@pytest.mark.parametrize("s", [1, 3])
def test_sector_equals_full_grid_with_8_fold_data(orc, centre, r_in, s):
    nr, r_out = 24, 1.4
    fs = _sector_fields(nr, s, r_in, r_out, seed=10 + s + centre)
    full = {k: np.ascontiguousarray(np.tile(v, (8, 1))) for k, v in fs.items()}
    dr = (r_out - r_in) / nr
    r0 = r_in + dr / 2
    dt = 0.35 * min(dr, r0 * (math.pi / 4 / s)) / 12.5  # Courant bound of the sector grid
    ms, _ = _run(orc, fs, nr, s, r_in, r_out, 1, centre, 30, dt)
    mf, _ = _run(orc, full, nr, 8 * s, r_in, r_out, 0, centre, 30, dt)
    for k in ("rho", "ur", "uth", "T", "lam"):
        for rot in range(8):  # every sector of the full grid equals the sector run
            np.testing.assert_allclose(mf[k][rot * s:(rot + 1) * s], ms[k], rtol=1e-11, atol=1e-12)


def test_disc_centre_keeps_a_state_at_rest(orc):
    """A uniform gas at rest in a disc sector with the centre rule stays at
    rest: the centre ghost mirrors f with the velocity reversed (i -> i+4)."""
    nr, s = 16, 1
    w = W.uniform_state(nr, s, 1.2, 0.0, 0.0, 1.1, 0.2, r_in=0.0, r_out=1.0)
    m, _ = _run(orc, w.fields, nr, s, 0.0, 1.0, 1, 1, 40, 0.2 * (1.0 / nr / 2) * (math.pi / 4) / 12.5)
    np.testing.assert_allclose(m["rho"], 1.2, atol=1e-13)
    np.testing.assert_allclose(m["ur"], 0.0, atol=1e-13)


def test_centre_rule_reverses_the_radial_velocity(orc):
    """With the centre rule, radial inflow at the centre is reflected: a
    converging flow piles up density at the centre (a reflecting symmetry
    axis), while an outflow ghost would let it pass."""
    nr, s = 40, 1
    w = W.uniform_state(nr, s, 1.0, 0.0, 0.0, 1.0, 0.0, r_in=0.0, r_out=1.0)
    w.fields["ur"] = np.full((s, nr), -0.3)
    dt = 0.3 * (1.0 / nr / 2) * (math.pi / 4) / 12.5
    mc, _ = _run(orc, w.fields, nr, s, 0.0, 1.0, 1, 1, 200, dt)
    assert mc["rho"][0, 0] > 1.05
    assert abs(mc["ur"][0, 0]) < 0.3


def test_lambda_front_crosses_the_centre_of_a_full_disc(orc):
    """Full 2 pi disc with the centre rule: the inner ghost of a lambda cell
    is the cell across the centre (row m + ntheta / 2, same radius).  In a
    uniform Cartesian flow u_x (uniform f, an exact steady state of the
    update) a lambda front x = x0 moves at u_x straight through the centre:
    once it has passed, the innermost cells downstream are burnt and the
    front on the +x axis (row 0) has moved u_x t."""
    nr, nth, ux, x0, t_end = 32, 32, 0.5, -0.25, 0.8
    w = W.uniform_state(nr, nth, 1.0, ux, 0.0, 1.0, 0.0, r_in=0.0, r_out=1.0)
    r, th = W.grid(nr, nth, 0.0, 1.0)
    w.fields["lam"] = np.ascontiguousarray(np.where(r * np.cos(th) < x0, 1.0, 0.0))
    dt = 0.4 * (0.5 / nr) * (2 * math.pi / nth) / 12.5     # innermost ring's arc
    n = int(round(t_end / dt))
    p = orc.make_params(nr=nr, ntheta=nth, r_in=0.0, r_out=1.0, dt=dt, tau=1e-3,
                        omega1=0.0, omega2=0.0, r_bc_inner=1)
    f, lam = orc.init(p, w.fields)
    for _ in range(n):
        f, lam, _ = orc.step(p, f, lam)
    m = orc.macro(p, f, lam)
    np.testing.assert_allclose(m["rho"], 1.0, atol=1e-12)            # the flow stays uniform
    prof = lam[0]                                                     # theta = 0: the +x axis
    assert prof[0] > 0.75
    k = np.nonzero(prof < 0.5)[0][0]
    xf = r[0, k - 1] + (0.5 - prof[k - 1]) / (prof[k] - prof[k - 1]) * (r[0, k] - r[0, k - 1])
    assert xf == pytest.approx(x0 + ux * n * dt, abs=2.0 / nr)
