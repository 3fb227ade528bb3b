"""Non-equilibrium manifestations on the GPU (dbm_noneq, Sec. II.E) against
the oracle's Delta*_m, and the paper's shock / rarefaction sign criterion."""
import json

import numpy as np
import pytest

from gpu_helpers import oracle_params
from paper_1308_0653_gb300 import dbm
from paper_1308_0653_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 2e-3)])
def test_noneq_matches_the_oracle(orc, precision, tol):
    """Same state (the GPU run exported after 60 steps is not used: the oracle
    runs its own 60 steps from the same initial fields); Delta* components
    relative to their largest magnitude."""
    w = W.explosion(128, 64, nsteps=60, seed=31, dt=2e-5)
    sim = dbm.Simulation(dict(w.params, precision=precision))
    sim.init_state(w.fields)
    sim.step(w.nsteps)
    got = sim.noneq()
    sim.close()
    p = oracle_params(orc, w)
    f, lam = orc.init(p, w.fields)
    for _ in range(w.nsteps):
        f, lam, _ = orc.step(p, f, lam)
    ref = orc.noneq(p, f)
    errs = {}
    for c, name in enumerate(dbm.NONEQ):
        scale = max(np.abs(ref[c]).max(), 1e-3 * np.abs(ref[[0, 2, 9, 11]]).max())
        errs[name] = float(np.abs(got[c] - ref[c]).max() / scale)
    print("NONEQ", precision, json.dumps(errs))
    for name, err in errs.items():
        assert err <= tol, (name, err)


def test_shock_and_rarefaction_signs_on_the_gpu():
    nr, nth = 1024, 8
    w = W.uniform_state(nr, nth, 1.0, 0.0, 0.0, 1.0, 0.0, r_in=100.0, r_out=101.0)
    r, th = W.grid(nr, nth, 100.0, 101.0)
    w.fields["rho"] = np.ascontiguousarray(np.where(r < 100.5, 2.0, 1.0))
    w.fields["T"] = np.ascontiguousarray(np.where(r < 100.5, 2.0, 1.0))
    sim = dbm.Simulation(dict(w.params, precision="fp32", dt=0.4 / nr / 12.5, tau=5e-4))
    sim.init_state(w.fields)
    sim.step(800)
    m = sim.moments()
    d = sim.noneq()
    sim.close()
    dudr = np.gradient(m["ur"][0], r[0])
    js, jr = int(np.argmin(dudr)), int(np.argmax(dudr))
    assert r[0, js] > 100.5 > r[0, jr]
    assert d[0, 0, js] > 0 > d[0, 0, jr]
    np.testing.assert_allclose(d[0] + d[2], 0.0, atol=1e-5 * np.abs(d[0]).max())
