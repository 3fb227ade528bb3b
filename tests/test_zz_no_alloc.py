"""dbm_totals_noalloc: conservation totals for callers that cannot provide
device scratch memory (they hold only raw pointers to a state someone else
owns, or run under an allocator that refuses new device allocations
mid-run).  Its reduction scratch is a static device array, so the call
allocates nothing.  Its totals must equal those of dbm_moments call after
call, read in place from a running simulation's padded buffer or from the
unpadded export layout, because every call rewrites the scratch rows it
reads.  This file is collected last, so a run that stops at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1308_0653_gb300 import dbm
from paper_1308_0653_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _entry():
    """The entry point through the C ABI, with its prototype."""
    L = dbm.lib()
    fn = L.dbm_totals_noalloc
    fn.argtypes = [ctypes.POINTER(dbm.DbmParams), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)
    return torch


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_totals_of_a_live_padded_state_equal_dbm_moments_on_two_calls_in_a_row(precision):
    """nr = 200 is not a multiple of 32: the live rows are padded to ld = 224,
    and the call reads the state where the simulation keeps it."""
    torch = _cuda()
    fn = _entry()
    w = W.explosion(200, 96, nsteps=0, seed=11, dt=2e-5)
    sim = dbm.Simulation(dict(w.params, precision=precision))
    sim.init_state(w.fields)
    stream = torch.cuda.current_stream()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for nsteps in (10, 25):  # two calls in a row, on two different states
        sim.step(nsteps)
        ref = sim.moments(totals=True)["totals"]
        d_f, _, ld = sim.state_device()
        assert ld == 224
        out.fill_(np.nan)
        rc = fn(ctypes.byref(sim.p), ctypes.c_void_p(d_f), ld, ctypes.c_void_p(out.data_ptr()),
                ctypes.c_void_p(stream.cuda_stream))
        assert rc == dbm.DBM_OK, dbm.strerror(rc)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-11, atol=1e-13)
    sim.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_totals_of_the_export_layout_equal_dbm_moments(precision):
    """ld = 0 reads the unpadded layout dbm_export_state writes."""
    torch = _cuda()
    fn = _entry()
    w = W.explosion(200, 96, nsteps=0, seed=12, dt=2e-5)
    sim = dbm.Simulation(dict(w.params, precision=precision))
    sim.init_state(w.fields)
    sim.step(7)
    ref = sim.moments(totals=True)["totals"]
    f, _, _ = sim.export_state()
    d_f = torch.from_numpy(f).cuda()
    out = torch.full((4,), np.nan, dtype=torch.float64, device="cuda")
    rc = fn(ctypes.byref(sim.p), ctypes.c_void_p(d_f.data_ptr()), 0, ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == dbm.DBM_OK, dbm.strerror(rc)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-11, atol=1e-13)
    sim.close()


def test_noalloc_at_the_row_limit_and_without_allocating():
    """ntheta = DBM_NOALLOC_MAX_ROWS (the largest state the static scratch
    holds) matches dbm_moments; after a first call, repeated calls leave the
    device's free memory unchanged (nothing allocated, nothing freed)."""
    torch = _cuda()
    fn = _entry()
    w = W.explosion(8, 16384, nsteps=0, seed=13, dt=1e-6)
    sim = dbm.Simulation(dict(w.params, precision="fp32"))
    sim.init_state(w.fields)
    sim.step(3)
    ref = sim.moments(totals=True)["totals"]
    d_f, _, ld = sim.state_device()
    out = torch.full((4,), np.nan, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert fn(ctypes.byref(sim.p), ctypes.c_void_p(d_f), ld, ctypes.c_void_p(out.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-11, atol=1e-13)
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        assert fn(ctypes.byref(sim.p), ctypes.c_void_p(d_f), ld, ctypes.c_void_p(out.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-11, atol=1e-13)
    sim.close()


def test_noalloc_rejects_states_beyond_the_static_scratch():
    fn = _entry()
    p = dbm.dbm_params_default()
    p.ntheta = 16385  # one row more than DBM_NOALLOC_MAX_ROWS
    rc = fn(ctypes.byref(p), ctypes.c_void_p(256), 0, ctypes.c_void_p(256), None)
    assert rc == dbm.DBM_ENOMEM
    p.ntheta = 64
    assert fn(ctypes.byref(p), None, 0, ctypes.c_void_p(256), None) == dbm.DBM_EINVAL
    assert fn(ctypes.byref(p), ctypes.c_void_p(256), p.nr - 1, ctypes.c_void_p(256), None) == dbm.DBM_EINVAL
