"""Cases run by tests/test_gpu_debug_build.py in a child process, once with
the release library and once with the checked one (DBM_DEBUG=1): ragged and
degenerate grids, a disc sector, a batch of uneven simulations, FP32 and FP64.
Writes every final state and status to the .npz file given as argument."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1308_0653_gb300 import dbm  # noqa: E402
from paper_1308_0653_gb300 import workloads as W  # noqa: E402


def main(out):
    import torch
    torch.cuda.set_device(0)
    res = {}
    cases = [("5x3", W.random_smooth(5, 3, seed=1, dt=1e-5), 0),
             ("130x16", W.random_smooth(130, 16, seed=2, dt=1e-5), 1),
             ("257x9", W.random_smooth(257, 9, seed=3, dt=1e-5), 4),
             ("disc", W.paper_implosion(nr=150), 0)]
    for prec in ("fp32", "fp64"):
        for name, w, rows in cases:
            sim = dbm.Simulation(dict(w.params, precision=prec, rows_per_item=rows))
            sim.init_state(w.fields)
            sim.step(40)
            f, lam, _ = sim.export_state()
            res[f"{name}_{prec}_f"], res[f"{name}_{prec}_lam"] = f, lam
            res[f"{name}_{prec}_status"] = np.array(dbm.dbm_status(sim.h))
            sim.close()
        ws = W.batch(3, seed=7, nsteps=0, nmin=40, nmax=200, precision=prec)
        b = dbm.Batch(4, 1 << 16, precision=prec)
        sims = []
        for slot, w in enumerate(ws):
            s = dbm.Simulation(dict(w.params, precision=prec))
            s.init_state(w.fields)
            b.attach(slot, s, 30 + 10 * slot)
            sims.append(s)
        b.step(60)
        for k, s in enumerate(sims):
            f, lam, _ = s.export_state()
            res[f"batch{k}_{prec}_f"], res[f"batch{k}_{prec}_lam"] = f, lam
            res[f"batch{k}_{prec}_status"] = np.array(dbm.dbm_status(s.h))
            s.close()
        b.close()
    res["library"] = np.array(dbm.lib_path())
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])
