"""Pins of the oracle's full time step (Sec. II.C-II.D, III.A) by invariants
and exact properties: uniform states, 8-fold rotation and mirror
equivariance of the Cartesian-fixed velocity set on a polar grid, the
direction and speed of pure advection, and upwind transport of lambda.
"""
import math
import os

import numpy as np
import pytest

from paper_1308_0653_gb300 import workloads as W


def _p(orc, w, **kw):
    d = {k: v for k, v in w.params.items() if k != "precision"}
    d.update(kw)
    return orc.make_params(**d)


@pytest.mark.parametrize("ux,uy,T", [(0.0, 0.0, 1.0), (0.3, -0.2, 1.2), (-0.8, 0.5, 2.0)])
def test_uniform_state_is_invariant(orc, ux, uy, T):
    """A spatially uniform state with f = f^eq has zero differences in every
    direction and is a fixed point of collision, so it stays put (any
    Cartesian velocity: its polar components vary with theta)."""
    w = W.uniform_state(16, 24, 1.3, ux, uy, T, 0.0, dt=1e-4)
    p = _p(orc, w)
    f, lam = orc.init(p, w.fields)
    for _ in range(20):
        f, lam, c = orc.step(p, f, lam)
        assert c == 0
    m = orc.macro(p, f, lam)
    for k in ("rho", "ur", "uth", "T", "lam"):
        np.testing.assert_allclose(m[k], w.fields[k], atol=1e-13, rtol=0)


def _rotate(f, lam, nth, shift_rows, dirs):
    """Rotate a state by shift_rows * dtheta with velocity directions i -> i + dirs."""
    g = np.empty_like(f)
    g[0] = np.roll(f[0], shift_rows, axis=0)
    for k in range(4):
        for i in range(8):
            g[1 + 8 * k + (i + dirs) % 8] = np.roll(f[1 + 8 * k + i], shift_rows, axis=0)
    return g, np.roll(lam, shift_rows, axis=0)


def _mirror(f, lam):
    """Reflect y -> -y: row m -> -m mod ntheta, direction i -> -i mod 8."""
    idx = (-np.arange(f.shape[1])) % f.shape[1]
    g = np.empty_like(f)
    g[0] = f[0][idx]
    for k in range(4):
        for i in range(8):
            g[1 + 8 * k + (-i) % 8] = f[1 + 8 * k + i][idx]
    return g, lam[idx]


def _random_state(orc, nr, nth, seed, **kw):
    w = W.random_smooth(nr, nth, seed=seed, amp=0.15, dt=2e-4, omega1=2.0, omega2=3.0, **kw)
    p = _p(orc, w)
    f, lam = orc.init(p, w.fields)
    # make f non-equilibrium so every term of the update is exercised
    rng = np.random.default_rng(seed)
    f = f * (1.0 + 0.01 * rng.standard_normal(f.shape))
    return p, f, lam


def test_rotation_by_pi_over_4_commutes_with_the_step(orc):
    """With ntheta a multiple of 8, rotating the state by pi/4 (rows shifted by
    ntheta/8, direction i -> i+1) commutes with one time step."""
    p, f, lam = _random_state(orc, 12, 32, seed=4)
    for _ in range(2):
        f1, l1, _ = orc.step(p, f, lam)
        fr, lr = _rotate(f, lam, 32, 4, 1)
        f2, l2, _ = orc.step(p, fr, lr)
        g1, m1 = _rotate(f1, l1, 32, 4, 1)
        np.testing.assert_allclose(f2, g1, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(l2, m1, rtol=1e-12, atol=1e-15)
        f, lam = f1, l1


def test_mirror_commutes_with_the_step(orc):
    """Reflection theta -> -theta (i -> -i) commutes with one time step."""
    p, f, lam = _random_state(orc, 10, 20, seed=5)
    f1, l1, _ = orc.step(p, f, lam)
    fm, lm = _mirror(f, lam)
    f2, l2, _ = orc.step(p, fm, lm)
    g1, m1 = _mirror(f1, l1)
    np.testing.assert_allclose(f2, g1, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(l2, m1, rtol=1e-12, atol=1e-15)


def test_axisymmetric_state_stays_axisymmetric_up_to_lattice_anisotropy(orc):
    """Axisymmetric data on a grid with ntheta = 8 q keep the 8-fold symmetry
    to round-off and stay theta-independent only up to the anisotropy of the
    8-direction velocity rings: on the 64 x 64 explosion the theta-variation
    of rho after 100 steps is 0.29 % and does not change when ntheta doubles
    (it is a property of the velocity set, not of the theta grid)."""
    w = W.explosion64()
    p = _p(orc, w)
    f, lam = orc.init(p, w.fields)
    for _ in range(100):
        f, lam, _ = orc.step(p, f, lam)
    m = orc.macro(p, f, lam)
    var = np.ptp(m["rho"], axis=0).max() / m["rho"].mean()
    assert var < 5e-3
    # exact 8-fold symmetry: rows m and m + ntheta/8 agree to round-off
    np.testing.assert_allclose(m["rho"], np.roll(m["rho"], 8, axis=0), rtol=1e-11)


def _centroid(p, f_q, r, th):
    x = r * np.cos(th)
    y = r * np.sin(th)
    w = f_q * r  # area element r dr dtheta (uniform dr, dtheta)
    return (w * x).sum() / w.sum(), (w * y).sum() / w.sum()


@pytest.mark.parametrize("k,i", [(1, 0), (2, 1), (1, 3), (3, 6)])
def test_pure_advection_moves_a_pulse_along_its_velocity(orc, k, i):
    """With no relaxation (tau -> inf, so exp(-dt/tau) = 1) and no reaction the
    update is pure upwind transport: a bump in one velocity channel moves with
    that channel's Cartesian velocity v_k (cos i pi/4, sin i pi/4), which fixes
    the sign of the streaming term and the geometry of C_r and C_theta."""
    nr, nth = 96, 256
    w = W.uniform_state(nr, nth, 1.0, 0.0, 0.0, 1.0, 0.0, r_in=0.5, r_out=1.5)
    vk = w.params["v"][k - 1]
    # dt from the fastest ring (12.5): |C_r| + |C_theta| < 1 for all 33 channels
    nsteps = int(math.ceil(0.12 / vk / (0.4 * min(1.0 / nr, 0.5 * 2 * math.pi / nth) / 12.5)))
    t_end = 0.12 / vk
    dt = t_end / nsteps
    p = _p(orc, w, dt=dt, tau=1e30)
    f, lam = orc.init(p, w.fields)
    r, th = W.grid(nr, nth, 0.5, 1.5)
    x0, y0 = 0.75, 0.45
    bump = 0.05 * np.exp(-((r * np.cos(th) - x0) ** 2 + (r * np.sin(th) - y0) ** 2) / (2 * 0.04 ** 2))
    q = 1 + 8 * (k - 1) + i
    base = f[q].copy()
    f[q] = f[q] + bump
    cx0, cy0 = _centroid(p, f[q] - base, r, th)
    for _ in range(nsteps):
        f, lam, _ = orc.step(p, f, lam)
    cx1, cy1 = _centroid(p, f[q] - base, r, th)
    ex = vk * math.cos(i * math.pi / 4) * t_end
    ey = vk * math.sin(i * math.pi / 4) * t_end
    cell = 1.0 / nr
    assert math.hypot(cx1 - cx0 - ex, cy1 - cy0 - ey) < cell, (cx1 - cx0, cy1 - cy0, ex, ey)
    # other channels did not move (differences in a uniform background are 0)
    others = [j for j in range(33) if j != q]
    f0, _ = orc.init(p, w.fields)
    np.testing.assert_allclose(f[others], f0[others], rtol=1e-12, atol=1e-15)


def test_lambda_is_carried_upwind_by_the_flow(orc):
    """Eq. (Eqlambda) transport part: a lambda front in a uniform outward flow
    (no reaction) moves outwards at u_r, to first order."""
    nr, nth = 200, 8
    w = W.uniform_state(nr, nth, 1.0, 0.0, 0.0, 1.0, 0.0, r_in=100.0, r_out=101.0)
    r, th = W.grid(nr, nth, 100.0, 101.0)
    u = 0.5
    w.fields["ur"] = np.full((nth, nr), u)
    w.fields["uth"] = np.zeros((nth, nr))
    w.fields["lam"] = np.ascontiguousarray(np.where(r < 100.3, 1.0, 0.0))
    dt = 0.4 * (1.0 / nr) / 12.5  # CFL of the fastest ring
    n = int(round(0.2 / u / dt))
    p = _p(orc, w, dt=dt, tau=1e-3)
    f, lam = orc.init(p, w.fields)
    for _ in range(n):
        f, lam, _ = orc.step(p, f, lam)
    # lambda = 1/2 crossing moved by u t
    prof = lam[0]
    j = np.nonzero(prof < 0.5)[0][0]
    xf = r[0, j - 1] + (0.5 - prof[j - 1]) / (prof[j] - prof[j - 1]) * (r[0, j] - r[0, j - 1])
    assert xf - 100.3 == pytest.approx(u * n * dt, abs=2.0 / nr)
    assert lam.min() >= 0.0 and lam.max() <= 1.0


def test_lambda_is_carried_upwind_in_theta(orc):
    """Eq. (Eqlambda) transport part in theta: on a thin annulus far from the
    axis (r = 100, locally a plane), a lambda front in a uniform azimuthal
    flow u_theta (no reaction) moves along theta by u_theta t of arc length,
    to first order, for either sign of u_theta."""
    nr, nth, r_in, r_out = 4, 2000, 100.0, 100.4
    r, th = W.grid(nr, nth, r_in, r_out)
    ds = r[0, 1] * (th[1, 0] - th[0, 0])               # arc length of a row at column 1
    dt = 0.4 * min((r_out - r_in) / nr, r_in * 2 * math.pi / nth) / 12.5
    for u in (0.5, -0.5):
        w = W.uniform_state(nr, nth, 1.0, 0.0, 0.0, 1.0, 0.0, r_in=r_in, r_out=r_out)
        w.fields["ur"] = np.zeros((nth, nr))
        w.fields["uth"] = np.full((nth, nr), u)
        w.fields["lam"] = np.ascontiguousarray(np.where(th < math.pi, 1.0, 0.0))
        n = int(round(5 * ds / abs(u) / dt))              # about five rows
        p = _p(orc, w, dt=dt, tau=1e-3)
        f, lam = orc.init(p, w.fields)
        for _ in range(n):
            f, lam, _ = orc.step(p, f, lam)
        prof = lam[:, 1]
        # the lambda = 1/2 crossing near theta = pi (rows 900 .. 1100)
        seg = prof[900:1100]
        k = 900 + np.nonzero(seg < 0.5)[0][0]
        x = (k - 1) + (0.5 - prof[k - 1]) / (prof[k] - prof[k - 1])
        moved = (x - (nth // 2 - 0.5)) * ds
        assert moved == pytest.approx(u * n * dt, abs=1.5 * ds), u
        assert lam.min() >= 0.0 and lam.max() <= 1.0


def test_outflow_boundary_lets_a_uniform_flow_through(orc):
    """Zero-gradient radial ghosts: a uniform radial-free flow (Cartesian
    uniform velocity) stays uniform at both radial boundaries."""
    w = W.uniform_state(8, 16, 0.9, 0.6, 0.0, 1.4, 0.5, dt=1e-4, r_in=0.5, r_out=1.0)
    p = _p(orc, w)
    f, lam = orc.init(p, w.fields)
    for _ in range(30):
        f, lam, _ = orc.step(p, f, lam)
    m = orc.macro(p, f, lam)
    np.testing.assert_allclose(m["rho"], 0.9, atol=1e-13)
    np.testing.assert_allclose(m["lam"], 0.5, atol=1e-13)


def test_bgk_relaxation_is_exact_exponential(orc):
    """Sec. II.C: the collision part is integrated analytically.  A uniform
    state with a moment-free non-equilibrium part delta relaxes as
    delta exp(-n dt / tau) (moments, hence f^eq, stay fixed)."""
    w = W.uniform_state(6, 16, 1.2, 0.2, -0.1, 1.3, 0.0, dt=1e-4, tau=7e-4)
    p = _p(orc, w)
    f, lam = orc.init(p, w.fields)
    feq = f.copy()
    # delta with zero mass, momentum and energy: (1, v, v^2) all vanish for a
    # combination of ring-2 and ring-3 opposite-direction pairs
    d = np.zeros(33)
    d[1 + 8 * 1 + 0] = d[1 + 8 * 1 + 4] = 1.0
    d[1 + 8 * 1 + 2] = d[1 + 8 * 1 + 6] = -1.0
    f = f + 1e-3 * d[:, None, None]
    n = 9
    for _ in range(n):
        f, lam, _ = orc.step(p, f, lam)
    expect = feq + 1e-3 * d[:, None, None] * math.exp(-n * 1e-4 / 7e-4)
    np.testing.assert_allclose(f, expect, rtol=0, atol=1e-14)


def test_streaming_is_consistent_with_v_dot_grad_on_linear_data(orc):
    """One step of pure streaming (tau -> inf, no reaction) on data linear in
    Cartesian x, y changes each channel by -dt v.grad f: exactly in r (cell
    centres r_j = r_in + (j + 1/2) dr) and to O(dtheta) in theta, where
    C_theta = v_th dt / (r_j dtheta) must use the same r_j as the data."""
    nr, nth = 8, 4096
    w = W.uniform_state(nr, nth, 1.0, 0.0, 0.0, 1.0, 0.0, r_in=1.0, r_out=2.0)
    dt = 0.4 * min(1.0 / nr, 2 * math.pi / nth) / 12.5
    p = _p(orc, w, dt=dt, tau=1e30)
    f, lam = orc.init(p, w.fields)
    r, th = W.grid(nr, nth, 1.0, 2.0)
    x, y = r * np.cos(th), r * np.sin(th)
    bx, by = 0.011, -0.007
    for q in range(1, 33):
        f[q] = f[q] + bx * x + by * y
    fn, _, _ = orc.step(p, f, lam)
    vk = np.repeat(np.array(w.params["v"]), 8)
    ang = np.tile(np.arange(8) * math.pi / 4, 4)
    for q in range(1, 33):
        expect = -dt * vk[q - 1] * (math.cos(ang[q - 1]) * bx + math.sin(ang[q - 1]) * by)
        got = (fn[q] - f[q])[:, 1:-1]  # interior columns (ghosts tested separately)
        np.testing.assert_allclose(got, expect, rtol=0, atol=2e-3 * abs(dt * vk[q - 1] * 0.013))


def test_radial_ghosts_are_zero_gradient(orc):
    """READING of the radial boundaries: the ghost at j = -1 (j = nr) copies
    j = 0 (j = nr - 1), so a channel whose upwind side is the ghost gets no
    radial change there, while interior sites get -C_r times the exact
    difference of data linear in r."""
    nr, nth = 10, 8
    w = W.uniform_state(nr, nth, 1.0, 0.0, 0.0, 1.0, 0.0, r_in=10.0, r_out=11.0)
    dt = 0.4 * (1.0 / nr) / 12.5
    p = _p(orc, w, dt=dt, tau=1e30)
    f, lam = orc.init(p, w.fields)
    r, th = W.grid(nr, nth, 10.0, 11.0)
    b = 0.02
    for q in range(1, 33):
        f[q] = f[q] + b * (r - 10.0)  # axisymmetric: theta differences vanish
    fn, _, _ = orc.step(p, f, lam)
    dr = 1.0 / nr
    for m in range(nth):
        vr, _ = orc.velocities(m * 2 * math.pi / nth, w.params["v"])
        for q in range(1, 33):
            Cr = vr[q] * dt / dr
            change = fn[q, m] - f[q, m]
            np.testing.assert_allclose(change[1:-1], -Cr * b * dr, atol=1e-15)
            if Cr > 1e-12:
                assert abs(change[0]) < 1e-15 and change[-1] == pytest.approx(-Cr * b * dr, abs=1e-15)
            elif Cr < -1e-12:
                assert abs(change[-1]) < 1e-15 and change[0] == pytest.approx(-Cr * b * dr, abs=1e-15)


@pytest.mark.parametrize("u", [-0.5, 0.5])
def test_lambda_radial_ghosts_are_zero_gradient(orc, u):
    """The radial ghosts of lambda copy the boundary cell (as for f): in a
    uniform radial flow u_r with lambda linear in r, the cell whose upwind
    side is the ghost keeps its lambda, and every other cell gains
    -u_r dt times the gradient."""
    nr, nth, b = 10, 8, 0.05
    w = W.uniform_state(nr, nth, 1.0, 0.0, 0.0, 1.0, 0.0, r_in=10.0, r_out=11.0)
    r, _ = W.grid(nr, nth, 10.0, 11.0)
    w.fields["ur"] = np.full((nth, nr), u)
    w.fields["uth"] = np.zeros((nth, nr))
    w.fields["lam"] = np.ascontiguousarray(0.3 + b * (r - 10.0))
    dt = 0.4 * (1.0 / nr) / 12.5
    p = _p(orc, w, dt=dt, tau=1e-3)
    f, lam = orc.init(p, w.fields)
    _, lam_n, _ = orc.step(p, f, lam)
    change = lam_n - lam
    edge, inner = (slice(-1, None), slice(None, -1)) if u < 0 else (slice(0, 1), slice(1, None))
    np.testing.assert_allclose(change[:, edge], 0.0, atol=1e-16)
    np.testing.assert_allclose(change[:, inner], -u * dt * b, rtol=1e-9)


def test_totals_are_area_weighted(orc):
    """Totals integrate with the area element r dr dtheta at cell centres
    (exact for fields linear in r): a uniform state has mass rho pi (r_out^2 -
    r_in^2), momentum rho pi (r_out^2 - r_in^2) (ux, uy) and energy
    rho (T + u^2/2) times the area.  The annulus' mean radius is 1.2, not 1,
    so an area element without r would give a different total."""
    w = W.uniform_state(7, 24, 1.3, 0.4, -0.2, 1.1, 0.0, r_in=0.3, r_out=2.1)
    p = _p(orc, w)
    f, lam = orc.init(p, w.fields)
    area = math.pi * (2.1 ** 2 - 0.3 ** 2)
    assert abs(area - 2 * math.pi * (2.1 - 0.3)) > 0.1 * area
    t = orc.totals(p, f)
    np.testing.assert_allclose(t, [1.3 * area, 1.3 * 0.4 * area, -1.3 * 0.2 * area,
                                   1.3 * (1.1 + 0.5 * (0.16 + 0.04)) * area], rtol=1e-13)


def _conserved(orc, p, f, lam):
    """Mass, momentum (polar components at each site's own theta) and total
    energy rho (T + u^2 / 2) densities (D = 2), per site."""
    m = orc.macro(p, f, lam)
    rho = m["rho"]
    return {"mass": rho, "mom_r": rho * m["ur"], "mom_th": rho * m["uth"],
            "energy": rho * (m["T"] + 0.5 * (m["ur"] ** 2 + m["uth"] ** 2))}, m


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_collision_conserves_mass_momentum_and_energy(orc, seed):
    """Sec. II.B-II.C: f^eq is built from the moments of f, so BGK relaxation
    keeps mass, momentum and energy at every site.  A spatially uniform f far
    from equilibrium (each velocity scaled by its own random factor, which
    changes all its moments) has no streaming differences: one step is the
    collision alone, and it moves f a long way while the conserved densities
    stay to round-off."""
    w = W.uniform_state(6, 16, 1.1, 0.25, -0.15, 1.4, 0.0, dt=1e-4, tau=3e-4)
    p = _p(orc, w)
    f, lam = orc.init(p, w.fields)
    rng = np.random.default_rng(100 + seed)
    f = f * (1.0 + rng.uniform(-0.3, 0.3, 33))[:, None, None]
    before, _ = _conserved(orc, p, f, lam)
    fn, lam_n, _ = orc.step(p, f, lam)
    after, _ = _conserved(orc, p, fn, lam_n)
    assert np.abs(fn - f).max() > 1e-3          # relaxed by far more than round-off
    for k in before:
        np.testing.assert_allclose(after[k], before[k], rtol=0, atol=2e-14, err_msg=k)


@pytest.mark.parametrize("mode", ["explicit", "consistent"])
def test_reaction_adds_exactly_the_heat_release(orc, mode):
    """Sec. II.A and III.A: the chemical term has no mass or momentum moment and
    an energy moment rho Q R.  One step of a uniform burning gas (T > T_th)
    keeps mass and momentum and adds dt rho Q R to the energy density, with
    R = (1 - lambda)(a + b lambda), a = omega1 P^m, b = omega2 P^n, P = rho T
    at time t (the printed equations); with the consistent reading
    R = (Lambda(lambda) - lambda) / dt the energy gained is exactly rho Q times
    the step's change of lambda."""
    rho, T, lam0, Q, w1, w2 = 1.1, 1.4, 0.3, 1.7, 2.0, 3.0
    w = W.uniform_state(6, 16, rho, 0.25, -0.15, T, lam0, dt=1e-4, tau=3e-4, omega1=w1,
                        omega2=w2, Q=Q)
    p = _p(orc, w, reaction_energy=mode)
    f, lam = orc.init(p, w.fields)
    before, _ = _conserved(orc, p, f, lam)
    fn, lam_n, _ = orc.step(p, f, lam)
    after, m = _conserved(orc, p, fn, lam_n)
    for k in ("mass", "mom_r", "mom_th"):
        np.testing.assert_allclose(after[k], before[k], rtol=0, atol=2e-14, err_msg=k)
    P = rho * T
    R = (1.0 - lam0) * (w1 * P + w2 * P * lam0)
    gain = rho * Q * (R * 1e-4 if mode == "explicit" else m["lam"] - lam0)
    assert np.all(m["lam"] > lam0)
    np.testing.assert_allclose(after["energy"] - before["energy"], gain, rtol=1e-10, atol=0)


def test_run_equals_repeated_steps(orc):
    """oracle.run (init, n steps and the moments in one call: the driver the
    GPU parity tests compare with) gives bit for bit what init, n separate
    steps and macro give, on a state where every term is active."""
    w = W.random_smooth(24, 16, seed=5, amp=0.15, dt=2e-4, omega1=2.0, omega2=3.0)
    p = _p(orc, w)
    n = 7
    out = orc.run(p, w.fields, n)
    f, lam = orc.init(p, w.fields)
    for _ in range(n):
        f, lam, _ = orc.step(p, f, lam)
    ref = orc.macro(p, f, lam)
    for k in ("rho", "ur", "uth", "T", "lam"):
        assert np.array_equal(out[k], ref[k]), k
    assert not np.array_equal(ref["rho"], w.fields["rho"])


def test_results_do_not_depend_on_the_thread_count(orc):
    """The oracle parallelises over theta rows only and each site is computed
    alone, so one thread and several give the same bits (the parity tests
    run it with however many cores the host has)."""
    w = W.random_smooth(40, 24, seed=8, amp=0.15, dt=2e-4, omega1=2.0, omega2=3.0)
    p = _p(orc, w)
    try:
        assert orc.set_threads(1) == 1
        one = orc.run(p, w.fields, 5)
        orc.set_threads(3)
        three = orc.run(p, w.fields, 5)
    finally:
        orc.set_threads(int(os.environ.get("ORACLE_THREADS", "0")))  # the session's setting
    for k in ("rho", "ur", "uth", "T", "lam"):
        assert np.array_equal(one[k], three[k]), k
