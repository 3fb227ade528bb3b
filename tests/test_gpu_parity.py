"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the
same seeded inputs: FP64 within 1e-11 and FP32 within 1e-4 relative L-inf,
on the paper-shaped workloads at oracle-friendly sizes, at full size for a
few steps in the benchmark's launch shape, and on ragged and degenerate grids.
"""
import numpy as np
import pytest

from gpu_helpers import FIELDS, TOL, assert_close, oracle_params, rel_errors, run_gpu, run_oracle
from paper_1308_0653_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_explosion64_full_run(orc, precision):
    """64 x 64 non-reactive explosion, 200 steps (the small FP64 config)."""
    w = W.explosion64()
    ref = run_oracle(orc, w)
    out = run_gpu(w, precision)
    assert_close(out, ref, TOL[precision], f"explosion64 {precision}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_reactive_explosion_128(orc, precision):
    """Reactive explosion (hot reacted ring, Cochran rate with ignition gate,
    1 % seeded density noise) on 128 x 128, 600 steps: every term active."""
    w = W.explosion(128, 128, nsteps=600, seed=0, dt=2e-5)
    ref = run_oracle(orc, w)
    assert ref["lam"].max() > 0.99 and ref["lam"].min() < 0.01
    out = run_gpu(w, precision)
    assert_close(out, ref, TOL[precision], f"explosion128 {precision}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_reactive_explosion_512_full(orc, precision):
    """The 512 x 512 reactive explosion for its full 5000 steps."""
    w = W.explosion(512, 512, nsteps=5000, seed=0)
    ref = run_oracle(orc, w)
    out = run_gpu(w, precision)
    assert_close(out, ref, TOL[precision], f"explosion512 {precision}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_implosion_2048_over_1000_steps_matches_the_oracle(orc, precision):
    """The 2048 x 2048 reactive implosion (the benchmark workload) for 1000
    steps, both precisions against the oracle run once for the module
    (1.4e11 site-velocity updates, about two minutes on 16 host cores): by
    then the fastest particles (speed 12.5) have crossed 128 cells and the
    driven shock about 15."""
    w = W.implosion(2048, 2048, nsteps=1000, seed=0)
    ref = run_oracle(orc, w)
    assert ((ref["lam"] > 0.01) & (ref["lam"] < 0.99)).any()
    out = run_gpu(w, precision)
    assert out["launch"]["grid"] == 304
    assert_close(out, ref, TOL[precision], f"implosion2048 1000 steps {precision}")


@pytest.mark.parametrize("omega1", [1.0, 2.0, 4.0])
def test_implosion_2048_in_bench_launch_shape(orc, omega1):
    """2048 x 2048 reactive implosion, FP32, 20 steps, for each of the rate
    constants omega1 in {1, 2, 4} of the workload definition, in the launch
    shape the benchmark times (automatic rows per item, persistent grid)."""
    w = W.implosion(2048, 2048, nsteps=20, seed=0, omega1=omega1)
    ref = run_oracle(orc, w)
    out = run_gpu(w, "fp32")
    assert out["launch"]["threads"] in (128, 160) and out["launch"]["grid"] == 304
    assert_close(out, ref, TOL["fp32"], f"implosion2048 omega1={omega1:g} fp32")


@pytest.mark.parametrize("nr,nth,rows", [(1, 8, 0), (5, 3, 0), (100, 7, 0), (130, 16, 1),
                                         (257, 9, 4), (33, 1, 0), (64, 2, 0), (96, 24, 1000),
                                         (200, 40, 3)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ragged_and_degenerate_grids(orc, nr, nth, rows, precision):
    """Ragged radial tails (nr not a multiple of the 128/64-site strip),
    ntheta not a multiple of 8 (direct angles), ntheta = 1 and 2 (a row is its
    own theta neighbour), nr = 1 (both radial ghosts), and forced rows per item."""
    w = W.random_smooth(nr, nth, seed=nr + nth, amp=0.1, r_in=0.5, r_out=1.5, omega1=3.0,
                        omega2=5.0, dt=2e-4, tau=5e-4)
    w.fields["T"] = w.fields["T"] * 0.9  # straddle the ignition temperature
    ref = run_oracle(orc, w, nsteps=25)
    out = run_gpu(w, precision, nsteps=25, rows_per_item=rows)
    assert_close(out, ref, TOL[precision], f"{nr}x{nth} rows={rows} {precision}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_consistent_reaction_energy_and_general_exponents(orc, precision):
    """Options: R taken as the step's lambda increment, and Cochran exponents
    m, n other than 1 (pow path)."""
    w = W.explosion(64, 32, nsteps=100, seed=3, dt=4e-5)
    ref = run_oracle(orc, w, reaction_energy=1, m=1.5, n=0.7)
    out = run_gpu(w, precision, reaction_energy=1, m=1.5, n=0.7)
    assert_close(out, ref, TOL[precision], f"consistent {precision}")


def test_totals_match_the_oracle(orc):
    w = W.explosion(96, 64, nsteps=50, seed=1, dt=2e-5)
    p = oracle_params(orc, w)
    f, lam = orc.init(p, w.fields)
    for _ in range(50):
        f, lam, _ = orc.step(p, f, lam)
    tot = orc.totals(p, f)
    out = run_gpu(w, "fp64")
    np.testing.assert_allclose(out["totals"], tot, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_uniform_state_stays_uniform(precision):
    """A uniform moving state is a fixed point of the update (every difference
    vanishes and f = f^eq), over 500 steps."""
    w = W.uniform_state(200, 64, 1.3, 0.3, -0.2, 1.2, 0.4, dt=1e-5)
    out = run_gpu(w, precision, nsteps=500)
    # FP32: 500 steps of round-off in f (a random walk of ~0.5 ulp per step)
    tol = 1e-12 if precision == "fp64" else 1e-5
    for k in FIELDS:
        np.testing.assert_allclose(out[k], w.fields[k], atol=tol * max(1.0, np.abs(w.fields[k]).max()))


def test_rotation_by_pi_over_4_fp32():
    """8-fold rotation equivariance on the GPU: rotating the initial data by
    pi/4 rotates the result (FP32, to round-off)."""
    w = W.random_smooth(64, 64, seed=9, amp=0.1, dt=2e-5, omega1=2.0, omega2=2.0)
    rot = W.Workload(w.name, w.params, {k: np.ascontiguousarray(np.roll(v, 8, axis=0))
                                        for k, v in w.fields.items()}, 0)
    a = run_gpu(w, "fp32", nsteps=100)
    b = run_gpu(rot, "fp32", nsteps=100)
    for k in FIELDS:
        np.testing.assert_allclose(np.roll(a[k], 8, axis=0), b[k], atol=2e-6, rtol=0)


def test_graph_and_single_launches_are_bitwise_identical():
    """dbm_step(n) replays a captured CUDA graph for runs of 32 steps; the
    result equals n single-step calls bit for bit."""
    from paper_1308_0653_gb300 import dbm
    w = W.explosion(160, 48, nsteps=0, seed=2, dt=2e-5)
    outs = []
    for chunks in ([70], [1] * 70):
        sim = dbm.Simulation(dict(w.params, precision="fp32"))
        sim.init_state(w.fields)
        for c in chunks:
            sim.step(c)
        assert dbm.dbm_steps_done(sim.h) == 70
        outs.append(sim.export_state())
        sim.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_zero_steps_is_a_noop(orc):
    w = W.explosion(32, 16, nsteps=0, seed=4)
    out = run_gpu(w, "fp64", nsteps=0)
    ref = run_oracle(orc, w, nsteps=0)
    assert_close(out, ref, TOL["fp64"], "zero steps")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_every_kernel_variant_gives_the_same_bits(precision):
    """The step-kernel variants differ only in staging (row barrier or
    producer warp, ring depth, registers); the update is bit for bit the same."""
    from paper_1308_0653_gb300 import dbm
    w = W.explosion(300, 72, nsteps=0, seed=12, dt=2e-5)
    states = []
    for v in range(1, dbm.dbm_num_variants(dbm.DBM_FP64 if precision == "fp64" else dbm.DBM_FP32) + 1):
        sim = dbm.Simulation(dict(w.params, precision=precision, variant=v))
        assert sim.launch_info()["variant"] == v
        sim.init_state(w.fields)
        sim.step(45)
        states.append(sim.export_state())
        sim.close()
    for f, lam, s in states[1:]:
        assert np.array_equal(f, states[0][0]) and np.array_equal(lam, states[0][1])


def _busiest_rows(ntheta, strips, slots, L):
    """Rows the busiest persistent CTA loads: items are dealt round-robin and
    each loads its L rows plus two halo rows."""
    items = strips * -(-ntheta // L)
    return -(-items // slots) * (L + 2)


@pytest.mark.parametrize("precision,n", [("fp32", 1536), ("fp32", 2048), ("fp32", 3072),
                                         ("fp64", 512), ("fp64", 2048)])
def test_work_items_balance_the_persistent_grid(precision, n):
    """The automatic rows per item leave the busiest CTA no more rows than
    any other choice would (brute force over every L here).  A choice from
    the average load alone, ceil(ntheta x strips / slots) rows, can give a
    few more items than CTAs: on 2048^2 FP64 it gave 320 items to 304 CTAs,
    so 16 of them ran two items and the step took twice the rows."""
    import torch
    from paper_1308_0653_gb300 import dbm
    w = W.implosion(64, 64, nsteps=0, seed=0)
    sim = dbm.Simulation(dict(w.params, nr=n, ntheta=n, precision=precision))
    info = sim.launch_info()
    sim.close()
    slots = 2 * torch.cuda.get_device_properties(0).multi_processor_count  # 2 CTAs per SM
    width = info["threads"] - 32                                           # producer warp + W sites
    strips = -(-n // width)
    L = info["rows_per_item"]
    assert info["items"] == strips * -(-n // L) and info["grid"] == min(info["items"], slots)
    assert (L, info["items"]) == dbm.dbm_plan_items(n, n, width, slots)
    best = min(_busiest_rows(n, strips, slots, c) for c in range(1, n + 1))
    assert _busiest_rows(n, strips, slots, L) == best


def test_work_items_in_several_waves_give_the_same_bits():
    """1536^2 FP64 runs 600 work items of 62 rows on 304 CTAs (two waves);
    one item per strip (1536 rows) gives the same bits."""
    from paper_1308_0653_gb300 import dbm
    w = W.explosion(1536, 1536, nsteps=0, seed=14)
    states = []
    for rows in (0, 1536):
        sim = dbm.Simulation(dict(w.params, precision="fp64", rows_per_item=rows))
        if rows == 0:
            assert sim.launch_info()["items"] > sim.launch_info()["grid"]
        sim.init_state(w.fields)
        sim.step(3)
        states.append(sim.export_state())
        sim.close()
    assert np.array_equal(states[0][0], states[1][0]) and np.array_equal(states[0][1], states[1][1])


def test_autotune_picks_a_variant_and_keeps_the_update(orc):
    from paper_1308_0653_gb300 import dbm
    w = W.explosion(256, 64, nsteps=0, seed=13, dt=2e-5)
    sim = dbm.Simulation(dict(w.params, precision="fp32"))
    sim.init_state(w.fields)
    best, ms = sim.autotune(steps=4)
    n = dbm.dbm_num_variants(dbm.DBM_FP32)
    assert 1 <= best <= n and all(x > 0 for x in ms[:n])
    assert sim.launch_info()["variant"] == best
    assert dbm.dbm_steps_done(sim.h) == n * 6
    sim.step(10)
    out = sim.moments()
    sim.close()
    ref = run_oracle(orc, w, nsteps=n * 6 + 10)
    assert_close(out, ref, TOL["fp32"], "after autotune")
    # the size class now defaults to the tuned variant
    sim2 = dbm.Simulation(dict(w.params, precision="fp32"))
    assert sim2.launch_info()["variant"] == best
    sim2.close()


def test_fp32_burning_completes_as_lambda_approaches_one(orc):
    """A hot gas at rest that is almost burnt (lambda = 1 - 1e-5) keeps
    burning in FP32 as in the FP64 oracle: 1 - lambda decays by e^-4 over
    1000 steps.  Per-step increments of lambda here (4e-8 down to 7e-10)
    are below the spacing of floats just under 1, so a lambda stored as a
    float would stall; the FP32 path stores 1 - lambda and tracks the oracle
    to 1e-3 relative in 1 - lambda itself."""
    w = W.uniform_state(32, 8, 1.0, 0.0, 0.0, 2.0, 1.0 - 1e-5, dt=1e-5, omega1=100.0, omega2=100.0)
    out = run_gpu(w, "fp32", nsteps=1000)
    ref = run_oracle(orc, w, nsteps=1000)
    y_gpu, y_ref = 1.0 - out["lam"], 1.0 - ref["lam"]
    assert y_ref.max() < 2.5e-7  # the oracle did burn
    np.testing.assert_allclose(y_gpu, y_ref, rtol=1e-3)


def test_implosion_2048_full_length_fp32_tracks_fp64():
    """The 2048 x 2048 implosion over its full 20 000 steps, FP32 against the
    FP64 GPU path (which matches the oracle to ~1e-13 on the parity cases; the
    oracle itself would need about 45 CPU-minutes for this run): every field
    within the FP32 target 1e-4 relative L-inf.  The FP32 reaction variable
    is rounded without bias; rounded to nearest, lambda fell 1.7e-4 behind."""
    w = W.implosion(2048, 2048, nsteps=20000, seed=0)
    a = run_gpu(w, "fp32")
    b = run_gpu(w, "fp64")
    assert_close(a, b, TOL["fp32"], "implosion2048 20000 steps fp32 vs fp64")


def test_large_grid_uniform_state_stays_uniform():
    """16384 x 8192 sites (36.5 GB of FP32 state): the offsets of the
    velocity planes pass 2^31 elements, the TMA row coordinates reach 8191,
    and the launch holds 2432 work items of 432 rows (8 per CTA).  A uniform
    moving state is a fixed point of the update, so after 4 steps every site
    still holds it (FP32)."""
    import torch
    nr, nth = 16384, 8192
    w = W.uniform_state(nr, nth, 1.3, 0.3, -0.2, 1.2, 0.4, r_in=1.0, r_out=2.0, dt=2e-6)
    free, _ = torch.cuda.mem_get_info()
    if free < 60e9:
        pytest.skip("needs about 40 GB of free device memory")
    out = run_gpu(w, "fp32", nsteps=4)
    assert out["launch"]["items"] == 2432 and out["launch"]["rows_per_item"] == 432
    for k in FIELDS:
        np.testing.assert_allclose(out[k], w.fields[k], atol=2e-6 * max(1.0, np.abs(w.fields[k]).max()))
