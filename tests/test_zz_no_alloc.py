"""dbm_totals_noalloc: conservation totals for callers that cannot provide
device scratch memory (they hold only raw pointers to a state someone else
owns, or run under an allocator that refuses new device allocations
mid-run).  Its reduction scratch is a static device array, so the call
allocates nothing; its totals must equal those of dbm_moments, call after
call, because every call rewrites the scratch rows it reads."""
import ctypes

import numpy as np
import pytest

from paper_1308_0653_gb300 import dbm
from paper_1308_0653_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _entry():
    L = dbm.lib()
    fn = L.dbm_totals_noalloc
    fn.argtypes = [ctypes.POINTER(dbm.DbmParams), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_totals_equal_dbm_moments_on_two_calls_in_a_row(precision):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)
    fn = _entry()
    w = W.explosion(200, 96, nsteps=0, seed=11, dt=2e-5)
    sim = dbm.Simulation(dict(w.params, precision=precision))
    sim.init_state(w.fields)
    stream = torch.cuda.current_stream()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for nsteps in (10, 25):  # two calls in a row on two different states
        sim.step(nsteps)
        ref = sim.moments(totals=True)["totals"]
        f, lam, _ = sim.export_state()
        d_f = torch.from_numpy(f).cuda()
        out.fill_(np.nan)
        rc = fn(ctypes.byref(sim.p), ctypes.c_void_p(d_f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                ctypes.c_void_p(stream.cuda_stream))
        assert rc == dbm.DBM_OK, dbm.strerror(rc)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-11, atol=1e-13)
    sim.close()


def test_noalloc_rejects_states_beyond_the_static_scratch():
    fn = _entry()
    p = dbm.dbm_params_default()
    p.ntheta = 16385  # one row more than DBM_NOALLOC_MAX_ROWS
    rc = fn(ctypes.byref(p), ctypes.c_void_p(256), ctypes.c_void_p(256), None)
    assert rc == dbm.DBM_ENOMEM
    p.ntheta = 64
    assert fn(ctypes.byref(p), None, ctypes.c_void_p(256), None) == dbm.DBM_EINVAL
