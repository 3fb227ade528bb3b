"""Shared helpers of the GPU tests: run a workload through the C ABI and
through the oracle, and compare fields by relative L-inf error.

Relative L-inf of a field: max |gpu - oracle| / scale with scale = max |oracle|
for rho, T and lambda (floored at 1e-12), and the largest oracle speed
max(|u_r|, |u_theta|) for both velocity components (they vanish in places),
floored at 1e-3 of the thermal speed sqrt(max T) (a state at rest has u = 0).
"""
import hashlib
import json

import numpy as np

FIELDS = ("rho", "ur", "uth", "T", "lam")

# Tolerances of the GPU path against the FP64 oracle: FP64 to 1e-11 and FP32 to
# 1e-4 relative L-inf after the run.
TOL = {"fp64": 1e-11, "fp32": 1e-4}


def rel_errors(gpu: dict, ref: dict) -> dict:
    out = {}
    # velocity floor: 1e-3 of the thermal speed (a state at rest has u = 0)
    uscale = max(np.abs(ref["ur"]).max(), np.abs(ref["uth"]).max(),
                 1e-3 * float(np.sqrt(np.abs(ref["T"]).max())))
    for k in FIELDS:
        if k in ("ur", "uth"):
            scale = uscale
        else:
            scale = max(np.abs(ref[k]).max(), 1e-12)
        out[k] = float(np.abs(gpu[k] - ref[k]).max() / scale)
    return out


def run_gpu(w, precision, nsteps=None, stream=None, **overrides):
    from paper_1308_0653_gb300 import dbm
    params = dict(w.params, precision=precision)
    params.update(overrides)
    sim = dbm.Simulation(params)
    try:
        sim.init_state(w.fields, stream=stream)
        sim.step(w.nsteps if nsteps is None else nsteps, stream=stream)
        out = sim.moments(stream=stream, totals=True)
        out["launch"] = sim.launch_info()
    finally:
        sim.close()
    return out


def oracle_params(orc, w, **overrides):
    d = {k: v for k, v in w.params.items() if k != "precision"}
    d.update({k: v for k, v in overrides.items() if k in d or k == "reaction_energy"})
    return orc.make_params(**d)


_ORACLE_CACHE = {}


def run_oracle(orc, w, nsteps=None, **overrides):
    """Oracle run of a workload (cached by parameters, step count, options and
    the bytes of the initial fields)."""
    n = w.nsteps if nsteps is None else nsteps
    digest = hashlib.sha1()
    for k in FIELDS:
        digest.update(np.ascontiguousarray(w.fields[k]).tobytes())
    key = (repr(sorted(w.params.items())), n, repr(sorted(overrides.items())), digest.hexdigest())
    if key not in _ORACLE_CACHE:
        p = oracle_params(orc, w, **overrides)
        _ORACLE_CACHE[key] = orc.run(p, w.fields, n)
    return _ORACLE_CACHE[key]


def assert_close(gpu, ref, tol, label=""):
    errs = rel_errors(gpu, ref)
    # one line per comparison, collected into the accuracy table from `pytest -s`
    print("ACCURACY", json.dumps({"case": label, "tol": tol, "errors": errs}))
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"{label}: relative L-inf above {tol}: {bad} (all: {errs})"
    return errs
