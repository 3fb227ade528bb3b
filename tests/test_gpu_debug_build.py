"""The checked build (DBM_DEBUG=1) adds device-side bounds and alignment
checks to every copy the producer warp issues and every store of the update
(compute-sanitizer stands in for nothing here: it is not available).  Run on
ragged grids, a disc sector and a batch, in FP32 and FP64, no check fires and
the results equal the release build's bit for bit (the checks read, never
change, the arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(out, debug):
    env = dict(os.environ)
    env.pop("DBM_DEBUG", None)
    if debug:
        env["DBM_DEBUG"] = "1"
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_cases.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    return dict(np.load(out))


def test_checked_build_is_clean_and_bitwise_equal_to_release(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    rel = _run(tmp_path / "release.npz", False)
    dbg = _run(tmp_path / "debug.npz", True)
    assert "_build_debug" in str(dbg["library"]) and "_build_debug" not in str(rel["library"])
    for k in rel:
        if k == "library":
            continue
        if k.endswith("_status"):
            assert int(dbg[k]) == 0 and int(rel[k]) == 0, k  # DBM_OK: no check fired
        else:
            assert np.array_equal(rel[k], dbg[k]), k
