"""The C ABI (include/dbm.h) without a GPU: the library loads, exports every
declared entry point, and its host-only calls (parameter checks, Courant
condition, buffer sizing) behave as documented."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1308_0653_gb300 import dbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(dbm_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_step_path_entry_points():
    names = declared_functions()
    for n in ("dbm_create", "dbm_init_state", "dbm_step", "dbm_moments", "dbm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = dbm.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", dbm.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (dbm_\w+)", out))
    assert set(declared_functions()) <= exported
    # the statically linked CUDA runtime stays private
    assert not re.search(r" T cuda[A-Z]", out)


def test_params_default_are_the_papers():
    p = dbm.dbm_params_default()
    assert list(p.v) == [1.5, 3.5, 7.5, 12.5]
    assert p.T_th == 1.1 and p.m == 1.0 and p.n == 1.0 and p.Q == 1.0
    assert p.precision == dbm.DBM_FP32
    assert dbm.strerror(dbm.DBM_ECFL).startswith("Courant")


def test_check_reports_the_courant_number():
    """max |C_r| + |C_theta| over velocities, rows and radii (Sec. II.C):
    the 12.5 ring at the innermost radius dominates."""
    p = dbm.dbm_params_default()
    st, cfl = dbm.dbm_check(p)
    assert st == dbm.DBM_OK
    dr = 1.0 / 64
    r0 = 0.05 + dr / 2
    dth = 2 * math.pi / 64
    best = max(12.5 * (abs(math.cos(a)) * 1e-5 / dr + abs(math.sin(a)) * 1e-5 / (r0 * dth))
               for a in [i * math.pi / 4 - m * dth for i in range(8) for m in range(64)])
    assert cfl == pytest.approx(best, rel=1e-12)
    p.dt = 1e-3
    st, cfl = dbm.dbm_check(p)
    assert st == dbm.DBM_ECFL and cfl > 1.0


@pytest.mark.parametrize("field,value", [("nr", 0), ("ntheta", -1), ("r_in", 0.0), ("r_out", 0.01),
                                         ("dt", 0.0), ("tau", 0.0), ("omega1", -1.0),
                                         ("precision", 7), ("reaction_energy", 3),
                                         ("rows_per_item", -2), ("variant", 99),
                                         ("variant", -1), ("sector", 2), ("reserved", 1),
                                         ("r_bc_inner", 1), ("r_bc_outer", 1), ("r_bc_inner", 7)])
def test_check_rejects_invalid_parameters(field, value):
    p = dbm.dbm_params_default()
    setattr(p, field, value)
    assert dbm.dbm_check(p)[0] == dbm.DBM_EINVAL
    assert dbm.dbm_state_bytes(p) == 0


def test_check_rejects_equal_ring_speeds():
    p = dbm.dbm_params_default()
    p.v[2] = p.v[1]
    assert dbm.dbm_check(p)[0] == dbm.DBM_EINVAL


def test_state_bytes_cover_both_buffers():
    """Two f buffers (33 planes) and two lambda buffers with rows padded to 32
    elements, in 4- or 8-byte words, plus small tables."""
    for prec, w in ((dbm.DBM_FP32, 4), (dbm.DBM_FP64, 8)):
        p = dbm.dbm_params_default()
        p.nr, p.ntheta, p.precision = 100, 40, prec
        ld = 128
        core = 2 * 34 * ld * 40 * w
        b = dbm.dbm_state_bytes(p)
        assert core <= b <= core + 64 * 1024 + 40 * 16 * w + ld * w


def test_create_validates_before_touching_the_gpu():
    p = dbm.dbm_params_default()
    h = ctypes.c_void_p()
    L = dbm.lib()
    assert L.dbm_create(ctypes.byref(p), None, 0, ctypes.byref(h)) == dbm.DBM_EINVAL
    p.dt = 1.0
    assert L.dbm_create(ctypes.byref(p), ctypes.c_void_p(256), 1 << 30, ctypes.byref(h)) == dbm.DBM_ECFL
    p = dbm.dbm_params_default()
    assert L.dbm_create(ctypes.byref(p), ctypes.c_void_p(256), 16, ctypes.byref(h)) == dbm.DBM_ENOMEM
    assert L.dbm_create(ctypes.byref(p), ctypes.c_void_p(100), 1 << 30, ctypes.byref(h)) == dbm.DBM_EINVAL


def test_null_handles_are_rejected():
    L = dbm.lib()
    assert L.dbm_step(None, 1, None) == dbm.DBM_EINVAL
    assert L.dbm_destroy(None) == dbm.DBM_EINVAL
    assert L.dbm_moments(None, None, None, None, None, None, None, None) == dbm.DBM_EINVAL
    assert L.dbm_steps_done(None) == -1


def test_variants_are_numbered_per_precision():
    for prec in (dbm.DBM_FP32, dbm.DBM_FP64):
        n = dbm.dbm_num_variants(prec)
        assert n >= 2
        p = dbm.dbm_params_default()
        p.precision = prec
        for v in range(0, n + 1):
            p.variant = v
            assert dbm.dbm_check(p)[0] == dbm.DBM_OK
        p.variant = n + 1
        assert dbm.dbm_check(p)[0] == dbm.DBM_EINVAL
    assert dbm.dbm_num_variants(7) == 0


def _busiest_rows(ntheta, strips, slots, rows):
    """Rows the busiest persistent CTA loads when items are dealt round-robin,
    each loading its rows plus two halo rows."""
    return -(-(strips * -(-ntheta // rows)) // slots) * (rows + 2)


@pytest.mark.parametrize("width,slots", [(128, 304), (64, 304), (96, 304), (128, 264)])
def test_plan_items_minimises_the_busiest_ctas_rows(width, slots):
    """dbm_plan_items, the split dbm_create uses, against brute force over
    every rows per item: the busiest CTA loads the fewest rows, and among the
    best choices the one with the fewest items (least halo traffic) wins."""
    for nr, nth in [(1, 1), (33, 1), (100, 7), (512, 512), (1536, 1536), (2048, 2048),
                    (3000, 517), (4096, 4096), (128, 20000)]:
        rows, items = dbm.dbm_plan_items(nr, nth, width, slots)
        strips = -(-nr // width)
        assert 1 <= rows <= nth and items == strips * -(-nth // rows)
        costs = [_busiest_rows(nth, strips, slots, L) for L in range(1, nth + 1)]
        best = min(costs)
        assert _busiest_rows(nth, strips, slots, rows) == best, (nr, nth)
        assert items == min(strips * -(-nth // L) for L in range(1, nth + 1) if costs[L - 1] == best)


def test_plan_items_cases_and_errors():
    # FP32 2048^2 (W = 128, 2 CTAs on each of 152 SMs): one wave of 304 items
    assert dbm.dbm_plan_items(2048, 2048, 128, 304) == (108, 304)
    # FP64 2048^2 (W = 64): 608 items, two per CTA.  The average-load rule
    # ceil(2048 x 32 / 304) = 216 rows gave 320 items, two for 16 CTAs only,
    # and twice the rows on the critical path.
    assert dbm.dbm_plan_items(2048, 2048, 64, 304) == (108, 608)
    assert (_busiest_rows(2048, 32, 304, 108), _busiest_rows(2048, 32, 304, 216)) == (220, 436)
    assert dbm.dbm_plan_items(1536, 1536, 64, 304) == (62, 600)
    # requested rows are kept, capped at ntheta
    assert dbm.dbm_plan_items(300, 72, 128, 304, 5) == (5, 3 * 15)
    assert dbm.dbm_plan_items(300, 72, 128, 304, 1000) == (72, 3)
    for bad in [(0, 8, 128, 304, 0), (8, 0, 128, 304, 0), (8, 8, 0, 304, 0), (8, 8, 128, 0, 0),
                (8, 8, 128, 304, -1)]:
        with pytest.raises(dbm.DbmError) as e:
            dbm.dbm_plan_items(*bad)
        assert e.value.status == dbm.DBM_EINVAL


def test_binding_checks_host_arrays_before_the_library_reads_them():
    """Host arrays reach the library as bare pointers, so the binding checks
    type, layout and size first (exceptions, not asserts)."""
    n = 12 * 7
    good = {k: np.zeros((12, 7)) for k in dbm.FIELDS}
    arrs = dbm._field_arrays(good, n)
    assert [a.size for a in arrs] == [n] * 5 and all(a.flags["C_CONTIGUOUS"] for a in arrs)
    ints = dict(good, T=np.ones((12, 7), dtype=np.int64))   # converted, not rejected
    assert dbm._field_arrays(ints, n)[3].dtype == np.float64
    with pytest.raises(ValueError):
        dbm._field_arrays(dict(good, lam=np.zeros((12, 6))), n)
    with pytest.raises(KeyError):
        dbm._field_arrays({k: v for k, v in good.items() if k != "uth"}, n)
    assert dbm._ptr(None) is None and dbm._ptr(np.zeros(4), 4) is not None
    with pytest.raises(ValueError):
        dbm._ptr(np.zeros(3), 4)
    with pytest.raises(TypeError):
        dbm._ptr(np.zeros(4, dtype=np.float32))
    with pytest.raises(TypeError):
        dbm._ptr(np.zeros((4, 4))[:, 1])                     # not contiguous
    with pytest.raises(ValueError):
        dbm.dbm_batch_plan([5, 6], [5], [1, 1], 128, 8, 100)
