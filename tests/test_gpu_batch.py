"""Batched execution: many uneven simulations advanced by one persistent
launch per step give, for each simulation, the same result as running it
alone (bit for bit: each site's update does not depend on how the grid is
cut into work items), including slots that join and leave mid-run."""
import numpy as np
import pytest

from gpu_helpers import TOL, assert_close, run_oracle
from paper_1308_0653_gb300 import dbm
from paper_1308_0653_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)


def _alone(w, precision, nsteps, variant=0):
    sim = dbm.Simulation(dict(w.params, precision=precision, variant=variant))
    sim.init_state(w.fields)
    sim.step(nsteps)
    st = sim.export_state()
    sim.close()
    return st


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_alone_bitwise(precision):
    ws = W.batch(6, seed=3, nsteps=0, nmin=40, nmax=300, precision=precision)
    steps = [37, 80, 5, 64, 1, 0]
    b = dbm.Batch(8, 4096, precision=precision, rows_per_item=7)
    sims = []
    for slot, (w, n) in enumerate(zip(ws, steps)):
        s = dbm.Simulation(dict(w.params, precision=precision))
        s.init_state(w.fields)
        b.attach(slot, s, n)
        sims.append(s)
    b.step(90)
    assert b.time() == 90
    # FP32 batches load rows through the slots' tensor maps; the reference
    # runs alone with per-array bulk copies (variant 2), so the comparison
    # also crosses the two ways of loading a row
    info = b.launch_info()
    assert info["variant"] == (4 if precision == "fp32" else 2)
    for s, w, n in zip(sims, ws, steps):
        assert dbm.dbm_steps_done(s.h) == n
        got = s.export_state()
        ref = _alone(w, precision, n, variant=2)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), w.name
    b.close()
    for s in sims:
        s.close()


def test_slots_join_and_leave_mid_run():
    """Continuous batching: a simulation attached after 40 steps and one
    detached after 20 both end where running alone would have put them."""
    ws = W.batch(3, seed=4, nsteps=0, nmin=64, nmax=200)
    b = dbm.Batch(4, 4096, rows_per_item=16)
    a = dbm.Simulation(dict(ws[0].params, precision="fp32"))
    a.init_state(ws[0].fields)
    c = dbm.Simulation(dict(ws[1].params, precision="fp32"))
    c.init_state(ws[1].fields)
    b.attach(0, a, 100)
    b.attach(1, c, 1000)
    b.step(20)
    b.detach(1)                        # c leaves after 20 steps
    b.step(20)
    d = dbm.Simulation(dict(ws[2].params, precision="fp32"))
    d.init_state(ws[2].fields)
    b.attach(1, d, 33)                 # d joins at T = 40 in the freed slot
    assert b.remaining(1) == 33
    b.step(70)
    assert b.remaining(0) == 0 and b.remaining(1) == 0
    for sim, w, n in ((a, ws[0], 100), (c, ws[1], 20), (d, ws[2], 33)):
        assert dbm.dbm_steps_done(sim.h) == n
        got = sim.export_state()
        ref = _alone(w, "fp32", n)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    b.close()
    for s in (a, c, d):
        s.close()


def test_batch_matches_the_oracle(orc):
    """Each member of a batch agrees with the FP64 oracle (FP32 tolerance)."""
    ws = W.batch(3, seed=5, nsteps=60, nmin=48, nmax=128)
    b = dbm.Batch(3, 4096)
    sims = []
    for slot, w in enumerate(ws):
        s = dbm.Simulation(dict(w.params, precision="fp32"))
        s.init_state(w.fields)
        b.attach(slot, s, w.nsteps)
        sims.append(s)
    b.step(60)
    for s, w in zip(sims, ws):
        assert_close(s.moments(), run_oracle(orc, w), TOL["fp32"], w.name)
        s.close()
    b.close()


def test_batch_rejects_mismatches():
    b = dbm.Batch(2, 3)
    w = W.explosion(64, 64, nsteps=0)
    s64 = dbm.Simulation(dict(w.params, precision="fp64"))
    with pytest.raises(dbm.DbmError):
        b.attach(0, s64, 5)            # precision differs
    s = dbm.Simulation(dict(w.params, precision="fp32"))
    s.init_state(w.fields)
    b.attach(0, s, 5)
    with pytest.raises(dbm.DbmError):
        b.attach(0, s, 5)              # slot taken
    with pytest.raises(dbm.DbmError) as e:
        b.step(1)                      # 1 strip x 4 row runs = 4 items > 3
    assert e.value.status == dbm.DBM_ENOMEM
    b.close()
    s.close()
    s64.close()


def test_batch_autotune_picks_a_kernel_and_keeps_the_update():
    """The batch autotuner times the default and bulk-copy kernels with 16, 32,
    64 and size-scaled rows per item on the live batch; the simulations it advanced end
    bit for bit where running alone for the same number of steps puts them."""
    ws = W.batch(4, seed=5, nsteps=0, nmin=64, nmax=300)
    b = dbm.Batch(4, 1 << 16, precision="fp32")
    sims = []
    for slot, w in enumerate(ws):
        s = dbm.Simulation(dict(w.params, precision="fp32"))
        s.init_state(w.fields)
        b.attach(slot, s, 1000)
        sims.append(s)
    v, r, ms = b.autotune(steps=8)
    assert v in (2, 4) and r in (16, 32, 64, -1)
    assert ms[0] > 0 and ms[4] > 0  # both kernels were timed
    info = b.launch_info()
    assert (info["variant"], info["rows_per_item"]) == (v, r)
    b.step(10)
    n = b.time()
    assert 10 < n <= 8 * (32 + 2 * 8) + 10
    for s, w in zip(sims, ws):
        assert dbm.dbm_steps_done(s.h) == n
        got = s.export_state()
        ref = _alone(w, "fp32", n, variant=2)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), w.name
    b.close()
    for s in sims:
        s.close()
