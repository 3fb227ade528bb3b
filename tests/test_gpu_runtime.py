"""Runtime behaviour of the C ABI on the GPU: checkpoint/resume, error
statuses made on the host (no GPU fault is ever provoked), streams."""
import numpy as np
import pytest

from paper_1308_0653_gb300 import dbm
from paper_1308_0653_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_checkpoint_resume_is_bitwise(precision):
    """Export after 37 steps, import into a fresh handle, run 40 more: equal
    bit for bit to 77 uninterrupted steps."""
    w = W.explosion(96, 40, nsteps=0, seed=5, dt=2e-5)
    a = dbm.Simulation(dict(w.params, precision=precision))
    a.init_state(w.fields)
    a.step(77)
    fa, la, sa = a.export_state()
    a.close()
    b = dbm.Simulation(dict(w.params, precision=precision))
    b.init_state(w.fields)
    b.step(37)
    f, lam, s = b.export_state()
    assert s == 37
    b.close()
    c = dbm.Simulation(dict(w.params, precision=precision))
    c.import_state(f, lam, s)
    c.step(40)
    fc, lc, sc = c.export_state()
    c.close()
    assert sc == sa == 77
    assert np.array_equal(fa, fc) and np.array_equal(la, lc)


def test_nonfinite_state_is_reported():
    """A NaN planted on the host (imported state) is reported by dbm_moments
    as DBM_ENONFINITE after a step, not as a crash."""
    w = W.explosion(64, 16, nsteps=0, seed=6)
    sim = dbm.Simulation(dict(w.params, precision="fp32"))
    sim.init_state(w.fields)
    f, lam, s = sim.export_state()
    f[3, 5, 7] = np.nan
    sim.import_state(f, lam, s)
    sim.step(2)
    out = sim.moments(raise_nonfinite=False)
    assert out["status"] == dbm.DBM_ENONFINITE
    assert np.isnan(out["rho"]).any()
    assert dbm.dbm_status(sim.h) == dbm.DBM_OK
    sim.close()


def test_invalid_initial_fields_are_rejected():
    w = W.explosion(32, 8, nsteps=0, seed=7)
    sim = dbm.Simulation(dict(w.params, precision="fp32"))
    bad = dict(w.fields)
    bad["T"] = bad["T"].copy()
    bad["T"][2, 3] = -1.0
    with pytest.raises(dbm.DbmError) as e:
        sim.init_state(bad)
    assert e.value.status == dbm.DBM_EINVAL
    bad["T"][2, 3] = np.inf
    with pytest.raises(dbm.DbmError):
        sim.init_state(bad)
    sim.close()


def test_buffer_too_small_and_courant_violation():
    import torch
    p = dbm.params_from(W.explosion(64, 64, nsteps=0).params)
    need = dbm.dbm_state_bytes(p)
    buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(dbm.DbmError) as e:
        dbm.dbm_create(p, buf.data_ptr(), need - 256)
    assert e.value.status == dbm.DBM_ENOMEM
    p.dt = 1e-3
    with pytest.raises(dbm.DbmError) as e:
        dbm.dbm_create(p, buf.data_ptr(), need)
    assert e.value.status == dbm.DBM_ECFL


def test_work_on_a_side_stream_matches_default_stream():
    import torch
    w = W.explosion(128, 64, nsteps=40, seed=8, dt=2e-5)
    a = dbm.Simulation(dict(w.params, precision="fp32"))
    a.init_state(w.fields)
    a.step(40)
    ra = a.moments()
    a.close()
    s = torch.cuda.Stream()
    b = dbm.Simulation(dict(w.params, precision="fp32"))
    b.init_state(w.fields, stream=s)
    b.step(40, stream=s)
    rb = b.moments(stream=s)
    b.close()
    for k in ("rho", "ur", "uth", "T", "lam"):
        assert np.array_equal(ra[k], rb[k])


def test_device_resident_init_and_moments(orc):
    """dbm_init_state_device / dbm_moments_device give the same result as the
    host-array calls."""
    import torch
    w = W.explosion(96, 32, nsteps=30, seed=9, dt=2e-5)
    host = dbm.Simulation(dict(w.params, precision="fp64"))
    host.init_state(w.fields)
    host.step(30)
    rh = host.moments()
    host.close()
    dev = dbm.Simulation(dict(w.params, precision="fp64"))
    fields = torch.from_numpy(np.stack([w.fields[k] for k in ("rho", "ur", "uth", "T", "lam")])).cuda()
    dbm.dbm_init_state_device(dev.h, fields.data_ptr())
    dbm.dbm_step(dev.h, 30)
    out = torch.empty_like(fields)
    dbm.dbm_moments_device(dev.h, out.data_ptr())
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    dev.close()
    for c, k in enumerate(("rho", "ur", "uth", "T", "lam")):
        assert np.array_equal(res[c], rh[k])


def test_fp32_reciprocal_is_within_one_ulp_of_ieee():
    """The FP32 step takes 1/rho, 1/T and the lambda-step denominator from the
    hardware reciprocal plus one Newton-Raphson step; over 10 decades of x it
    stays within 1 ulp of the correctly rounded 1/x."""
    import ctypes
    import torch
    L = dbm.lib()
    L.dbm_selftest_rcp.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]
    g = torch.Generator().manual_seed(0)
    x = torch.exp(torch.empty(1 << 20).uniform_(-12.0, 11.0, generator=g)).float().cuda()
    a, b = torch.empty_like(x), torch.empty_like(x)
    assert L.dbm_selftest_rcp(x.data_ptr(), a.data_ptr(), b.data_ptr(), x.numel(), None) == 0
    torch.cuda.synchronize()
    ulp = (a.view(torch.int32).long() - b.view(torch.int32).long()).abs()
    assert int(ulp.max()) <= 1


def test_bounded_wait_runs_out_reports_and_leaves_the_context_usable():
    """The device waits of the step kernels give up after a cycle limit: a
    wait on an mbarrier that nothing arrives on ends after 2^22 cycles (about
    2 ms) with the timeout bit set, the context still runs kernels, and the
    same wait with an arrival completes without it."""
    import torch
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    dbm.dbm_selftest_wait(st.data_ptr(), False, 1 << 22)        # nothing arrives
    dbm.dbm_selftest_wait(st.data_ptr() + 4, True, 1 << 22)     # warp 1 arrives
    torch.cuda.synchronize()
    assert st.tolist() == [1, 0]
    # the context is intact: a step runs and is finite
    w = W.explosion(64, 32, nsteps=0, seed=3)
    out = dbm.Simulation(dict(w.params, precision="fp32"))
    out.init_state(w.fields)
    out.step(5)
    m = out.moments()
    assert np.isfinite(m["rho"]).all() and dbm.dbm_status(out.h) == dbm.DBM_OK
    out.close()
    with pytest.raises(Exception):
        dbm.dbm_selftest_wait(st.data_ptr(), False, 0)          # invalid limit


def test_device_init_check_is_reported_by_status_and_cleared_by_a_good_init():
    """dbm_init_state_device checks the fields on the GPU without waiting: a
    bad value is reported by the next dbm_status as DBM_EINVAL, and a later
    init with valid fields clears it."""
    import torch
    w = W.explosion(64, 16, nsteps=0, seed=10)
    sim = dbm.Simulation(dict(w.params, precision="fp32"))
    fields = np.stack([w.fields[k] for k in ("rho", "ur", "uth", "T", "lam")])
    bad = fields.copy()
    bad[0, 3, 5] = 0.0                                   # rho = 0
    d_bad = torch.from_numpy(bad).cuda()
    dbm.dbm_init_state_device(sim.h, d_bad.data_ptr())
    assert dbm.dbm_status(sim.h) == dbm.DBM_EINVAL
    bad[0, 3, 5] = np.nan
    d_bad.copy_(torch.from_numpy(bad))
    dbm.dbm_init_state_device(sim.h, d_bad.data_ptr())
    assert dbm.dbm_status(sim.h) == dbm.DBM_EINVAL
    d_good = torch.from_numpy(fields).cuda()
    dbm.dbm_init_state_device(sim.h, d_good.data_ptr())
    assert dbm.dbm_status(sim.h) == dbm.DBM_OK
    sim.close()


def test_destroy_waits_for_the_handles_queued_steps():
    """dbm_destroy returns only after the GPU has finished the steps queued
    on the handle's buffers: the stream they were queued on is idle then."""
    import torch
    w = W.implosion(1024, 1024, nsteps=0)
    p = dbm.params_from(dict(w.params, precision="fp32"))
    need = dbm.dbm_state_bytes(p)
    buf = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    ptr = (buf.data_ptr() + 255) // 256 * 256
    h = dbm.dbm_create(p, ptr, need)
    s = torch.cuda.Stream()
    dbm.dbm_init_state(h, *[w.fields[k] for k in ("rho", "ur", "uth", "T", "lam")], stream=s)
    dbm.dbm_step(h, 400, s)                              # about 20 ms of work
    assert not s.query()                                 # still running
    dbm.dbm_destroy(h)
    assert s.query()                                     # finished before destroy returned


def test_batches_share_the_constant_table_and_give_entries_back():
    """Every live batch holds max_slots entries of the per-precision constant
    table (256 FP32 entries per device): a batch that does not fit is refused
    with DBM_ENOMEM, and a destroyed batch's entries can be taken again."""
    import gc
    gc.collect()                                         # batches of earlier tests
    a = dbm.Batch(200, 1024, precision="fp32")
    with pytest.raises(dbm.DbmError) as e:
        dbm.Batch(100, 1024, precision="fp32")
    assert e.value.status == dbm.DBM_ENOMEM
    b = dbm.Batch(56, 1024, precision="fp32")            # 200 + 56 = 256: fits
    a.close()
    c = dbm.Batch(150, 1024, precision="fp32")
    c.close()
    b.close()
    d = dbm.Batch(256, 1024, precision="fp32")
    d.close()


def test_two_handles_on_two_streams_interleaved_match_serial_solves():
    """A stream of solves through two handles on two streams, each solve's
    upload and its predecessor's download overlapping the other handle's
    steps (how the end-to-end throughput is measured).  512 x 512 FP32 states
    are 35 MB per buffer, so the host paths split into row chunks on each
    handle's second stream.  Every solve's fields equal, bit for bit, those of
    the same solve run alone."""
    import torch
    cases = [("explosion", 1, 12), ("implosion", 2, 7), ("explosion", 3, 9), ("implosion", 4, 5)]

    def work(kind, seed):
        f = W.explosion if kind == "explosion" else W.implosion
        return f(512, 512, nsteps=0, seed=seed)

    ref = []
    for kind, seed, n in cases:
        w = work(kind, seed)
        s = dbm.Simulation(dict(w.params, precision="fp32"))
        s.init_state(w.fields)
        s.step(n)
        ref.append(s.moments())
        s.close()
    sims = [dbm.Simulation(dict(work("explosion", 1).params, precision="fp32")),
            dbm.Simulation(dict(work("implosion", 2).params, precision="fp32"))]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    got = [None] * len(cases)
    for i in range(len(cases) + 1):
        if i < len(cases):
            kind, seed, n = cases[i]
            sims[i % 2].init_state(work(kind, seed).fields, stream=streams[i % 2])
            sims[i % 2].step(n, stream=streams[i % 2])
        if i > 0:
            got[i - 1] = sims[(i - 1) % 2].moments(stream=streams[(i - 1) % 2])
    for s in sims:
        s.close()
    for (kind, seed, n), g, r in zip(cases, got, ref):
        for k in dbm.FIELDS:
            assert np.array_equal(g[k], r[k]), (kind, seed, n, k)
