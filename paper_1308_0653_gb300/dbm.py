"""ctypes binding of the C ABI in include/dbm.h (argument marshalling only).

Every step of the update runs in the CUDA library ``libdbm.so``; this module
only converts arguments.  A missing or unloadable library raises; there is no
CPU fallback.  PyTorch supplies device memory (a uint8 tensor borrowed by the
library) and streams (``torch.cuda.Stream.cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

NV = 33
DBM_OK, DBM_EINVAL, DBM_ECFL, DBM_ENOMEM, DBM_EBUSY, DBM_ENOTREADY = 0, 1, 2, 3, 4, 5
DBM_ETIMEOUT, DBM_ENONFINITE, DBM_ECUDA, DBM_ECANCELLED, DBM_ENOTFOUND, DBM_EDEVICE = 6, 7, 8, 9, 10, 11
DBM_FP32, DBM_FP64 = 0, 1
DBM_BC_OUTFLOW, DBM_BC_CENTRE = 0, 1
DBM_R_EXPLICIT, DBM_R_CONSISTENT = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)


class DbmParams(ctypes.Structure):
    """Mirror of ``dbm_params``."""
    _fields_ = [
        ("nr", ctypes.c_int32), ("ntheta", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("reaction_energy", ctypes.c_int32),
        ("r_bc_inner", ctypes.c_int32), ("r_bc_outer", ctypes.c_int32),
        ("rows_per_item", ctypes.c_int32), ("variant", ctypes.c_int32),
        ("sector", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("r_in", ctypes.c_double), ("r_out", ctypes.c_double),
        ("dt", ctypes.c_double), ("tau", ctypes.c_double),
        ("Q", ctypes.c_double), ("omega1", ctypes.c_double), ("omega2", ctypes.c_double),
        ("m", ctypes.c_double), ("n", ctypes.c_double), ("T_th", ctypes.c_double),
        ("v", ctypes.c_double * 4),
    ]


class DbmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


_lib = None


def lib_path() -> str:
    return _build.LIB_DEBUG if _build.debug_requested() else _build.LIB


def lib():
    """Load libdbm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(DbmParams)
        H = ctypes.c_void_p
        vp = ctypes.c_void_p
        L.dbm_version.restype = ctypes.c_char_p
        L.dbm_strerror.argtypes = [ctypes.c_int]
        L.dbm_strerror.restype = ctypes.c_char_p
        L.dbm_last_error.restype = ctypes.c_char_p
        L.dbm_params_default.argtypes = [P]
        L.dbm_check.argtypes = [P, _dp]
        L.dbm_state_bytes.argtypes = [P]
        L.dbm_state_bytes.restype = ctypes.c_size_t
        L.dbm_plan_items.argtypes = [ctypes.c_int32] * 5 + [ctypes.POINTER(ctypes.c_int32),
                                                            ctypes.POINTER(ctypes.c_int64)]
        L.dbm_create.argtypes = [P, vp, ctypes.c_size_t, ctypes.POINTER(H)]
        L.dbm_destroy.argtypes = [H]
        L.dbm_init_state.argtypes = [H] + [_dp] * 5 + [vp]
        L.dbm_init_state_device.argtypes = [H, vp, vp]
        L.dbm_step.argtypes = [H, ctypes.c_int64, vp]
        L.dbm_moments.argtypes = [H] + [_dp] * 6 + [vp]
        L.dbm_moments_device.argtypes = [H, vp, vp]
        L.dbm_steps_done.argtypes = [H]
        L.dbm_steps_done.restype = ctypes.c_int64
        L.dbm_state_device.argtypes = [H, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64)]
        L.dbm_totals_noalloc.argtypes = [P, vp, ctypes.c_int64, vp, vp]
        L.dbm_status.argtypes = [H, vp]
        L.dbm_export_state.argtypes = [H, vp, vp, ctypes.POINTER(ctypes.c_int64), vp]
        L.dbm_import_state.argtypes = [H, vp, vp, ctypes.c_int64, vp]
        L.dbm_launch_info.argtypes = [H] + [ctypes.POINTER(ctypes.c_int)] * 6
        L.dbm_noneq.argtypes = [H, _dp, vp]
        L.dbm_noneq_device.argtypes = [H, vp, vp]
        L.dbm_selftest_wait.argtypes = [vp, ctypes.c_int, ctypes.c_int64, vp]
        L.dbm_num_variants.argtypes = [ctypes.c_int]
        L.dbm_set_variant.argtypes = [H, ctypes.c_int]
        L.dbm_autotune.argtypes = [H, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_float)]
        B = ctypes.c_void_p
        L.dbm_batch_bytes.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int]
        L.dbm_batch_bytes.restype = ctypes.c_size_t
        _ip = ctypes.POINTER(ctypes.c_int32)
        L.dbm_batch_plan.argtypes = [ctypes.c_int32, _ip, _ip, _ip, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int64, _ip, ctypes.POINTER(ctypes.c_int64)]
        L.dbm_batch_create.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp,
                                       ctypes.c_size_t, ctypes.POINTER(B)]
        L.dbm_batch_destroy.argtypes = [B]
        L.dbm_batch_attach.argtypes = [B, ctypes.c_int, H, ctypes.c_int64]
        L.dbm_batch_detach.argtypes = [B, ctypes.c_int]
        L.dbm_batch_remaining.argtypes = [B, ctypes.c_int]
        L.dbm_batch_remaining.restype = ctypes.c_int64
        L.dbm_batch_time.argtypes = [B]
        L.dbm_batch_time.restype = ctypes.c_int64
        L.dbm_batch_commit.argtypes = [B, vp]
        L.dbm_batch_step.argtypes = [B, ctypes.c_int64, vp]
        L.dbm_batch_launch_info.argtypes = [B] + [ctypes.POINTER(ctypes.c_int)] * 4
        L.dbm_batch_autotune.argtypes = [B, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().dbm_strerror(int(status)).decode()


def _check(status: int, where: str):
    if status != DBM_OK:
        raise DbmError(status, where)


def _ptr(a, size=None):
    """double* of a C-contiguous float64 array (None passes through); with
    `size`, the array must hold exactly that many elements, since the library
    reads or writes that many."""
    if a is None:
        return None
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous float64 numpy array")
    if size is not None and a.size != size:
        raise ValueError(f"array of {a.size} elements where {size} are needed")
    return a.ctypes.data_as(_dp)


def _field_arrays(fields, n: int):
    """The five host fields (rho, u_r, u_theta, T, lambda) as contiguous
    float64 arrays of n = ntheta x nr elements each (copies only if needed)."""
    arrs = [np.ascontiguousarray(fields[k], dtype=np.float64) for k in FIELDS]
    for k, a in zip(FIELDS, arrs):
        if a.size != n:
            raise ValueError(f"field {k}: {a.size} values for a grid of {n} sites")
    return arrs


def _stream(stream):
    """cudaStream_t value of a torch stream, an int handle, or None (default)."""
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ---- raw C-ABI entry points (same names) ----------------------------------

def dbm_version() -> str:
    return lib().dbm_version().decode()


def dbm_params_default() -> DbmParams:
    p = DbmParams()
    _check(lib().dbm_params_default(ctypes.byref(p)), "dbm_params_default")
    return p


def dbm_check(p: DbmParams):
    """Returns (status, max Courant sum)."""
    cfl = ctypes.c_double(0.0)
    st = lib().dbm_check(ctypes.byref(p), ctypes.byref(cfl))
    return st, cfl.value


def dbm_state_bytes(p: DbmParams) -> int:
    return int(lib().dbm_state_bytes(ctypes.byref(p)))


def dbm_batch_plan(nr, ntheta, rows_per_item, width: int, grid: int, max_items: int):
    """Host-only work items of a batched step: int32 array (n, 4) of (slot,
    first radial site, first theta row, end row), slot -1 for padding; CTA c
    runs rows c, c + grid, ...  nr[s] = 0 marks an empty slot."""
    nr, ntheta, rows = (np.ascontiguousarray(a, dtype=np.int32) for a in (nr, ntheta, rows_per_item))
    if not nr.shape == ntheta.shape == rows.shape or nr.ndim != 1:
        raise ValueError("nr, ntheta and rows_per_item must be 1-D arrays of one length")
    items = np.zeros((max_items, 4), dtype=np.int32)
    n = ctypes.c_int64(0)
    ip = ctypes.POINTER(ctypes.c_int32)
    _check(lib().dbm_batch_plan(len(nr), nr.ctypes.data_as(ip), ntheta.ctypes.data_as(ip),
                                rows.ctypes.data_as(ip), width, grid, max_items,
                                items.ctypes.data_as(ip), ctypes.byref(n)), "dbm_batch_plan")
    return items[:n.value].copy()


def dbm_plan_items(nr: int, ntheta: int, width: int, slots: int, rows_requested: int = 0):
    """Host-only work split of one simulation: (rows per item, items per step)."""
    rows, items = ctypes.c_int32(0), ctypes.c_int64(0)
    _check(lib().dbm_plan_items(nr, ntheta, width, slots, rows_requested, ctypes.byref(rows),
                                ctypes.byref(items)), "dbm_plan_items")
    return rows.value, items.value


def dbm_create(p: DbmParams, dev_ptr: int, nbytes: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().dbm_create(ctypes.byref(p), ctypes.c_void_p(dev_ptr), ctypes.c_size_t(nbytes),
                            ctypes.byref(h)), "dbm_create")
    return h


def dbm_destroy(h):
    _check(lib().dbm_destroy(h), "dbm_destroy")


def dbm_init_state(h, rho, ur, uth, T, lam, stream=None):
    """Host fields of the handle's grid (their sizes are the caller's to get
    right here; Simulation.init_state checks them against the grid)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ur, uth, T, lam)]
    if len({a.size for a in arrs}) != 1:
        raise ValueError("the five fields differ in size")
    _check(lib().dbm_init_state(h, *[_ptr(a) for a in arrs], _stream(stream)), "dbm_init_state")


def dbm_init_state_device(h, dev_fields_ptr: int, stream=None):
    _check(lib().dbm_init_state_device(h, ctypes.c_void_p(dev_fields_ptr), _stream(stream)),
           "dbm_init_state_device")


def dbm_step(h, nsteps: int, stream=None):
    _check(lib().dbm_step(h, int(nsteps), _stream(stream)), "dbm_step")


def dbm_moments(h, rho=None, ur=None, uth=None, T=None, lam=None, totals=None, stream=None,
                raise_nonfinite=True):
    st = lib().dbm_moments(h, _ptr(rho), _ptr(ur), _ptr(uth), _ptr(T), _ptr(lam), _ptr(totals, 4),
                           _stream(stream))
    if st == DBM_ENONFINITE and not raise_nonfinite:
        return st
    _check(st, "dbm_moments")
    return st


def dbm_moments_device(h, dev_out_ptr: int, stream=None):
    _check(lib().dbm_moments_device(h, ctypes.c_void_p(dev_out_ptr), _stream(stream)),
           "dbm_moments_device")


NONEQ = ("d2_rr", "d2_rth", "d2_thth", "d3_rrr", "d3_rrth", "d3_rthth", "d3_ththth",
         "d31_r", "d31_th", "d42_rr", "d42_rth", "d42_thth")


def dbm_noneq(h, out, stream=None):
    _check(lib().dbm_noneq(h, _ptr(out), _stream(stream)), "dbm_noneq")


def dbm_noneq_device(h, dev_out_ptr: int, stream=None):
    _check(lib().dbm_noneq_device(h, ctypes.c_void_p(dev_out_ptr), _stream(stream)),
           "dbm_noneq_device")


def dbm_steps_done(h) -> int:
    return int(lib().dbm_steps_done(h))


def dbm_state_device(h):
    """Device addresses of the current state in the handle's buffer and its
    row stride: (f address, lambda address, ld)."""
    f, lam, ld = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64(0)
    _check(lib().dbm_state_device(h, ctypes.byref(f), ctypes.byref(lam), ctypes.byref(ld)),
           "dbm_state_device")
    return f.value, lam.value, ld.value


def dbm_totals_noalloc(p: DbmParams, dev_f_ptr: int, ld: int, dev_totals_ptr: int, stream=None) -> int:
    """Enqueue the allocation-free totals of f[33][ntheta][ld] at dev_f_ptr
    into 4 device doubles at dev_totals_ptr; returns the status."""
    return int(lib().dbm_totals_noalloc(ctypes.byref(p), ctypes.c_void_p(dev_f_ptr), int(ld),
                                        ctypes.c_void_p(dev_totals_ptr), _stream(stream)))


def dbm_status(h, stream=None) -> int:
    return int(lib().dbm_status(h, _stream(stream)))


def dbm_export_state(h, f, lam, stream=None) -> int:
    steps = ctypes.c_int64(0)
    _check(lib().dbm_export_state(h, f.ctypes.data_as(ctypes.c_void_p),
                                  lam.ctypes.data_as(ctypes.c_void_p), ctypes.byref(steps),
                                  _stream(stream)), "dbm_export_state")
    return steps.value


def dbm_import_state(h, f, lam, steps: int, stream=None):
    _check(lib().dbm_import_state(h, f.ctypes.data_as(ctypes.c_void_p),
                                  lam.ctypes.data_as(ctypes.c_void_p), int(steps),
                                  _stream(stream)), "dbm_import_state")


def dbm_launch_info(h) -> dict:
    vals = [ctypes.c_int(0) for _ in range(6)]
    _check(lib().dbm_launch_info(h, *[ctypes.byref(v) for v in vals]), "dbm_launch_info")
    return dict(zip(("grid", "threads", "smem_bytes", "rows_per_item", "items", "variant"),
                    [v.value for v in vals]))


def dbm_selftest_wait(dev_status_ptr: int, arrive: bool, limit_cycles: int, stream=None):
    _check(lib().dbm_selftest_wait(ctypes.c_void_p(dev_status_ptr), int(bool(arrive)), int(limit_cycles),
                                   _stream(stream)), "dbm_selftest_wait")


def dbm_num_variants(precision: int) -> int:
    return int(lib().dbm_num_variants(int(precision)))


def dbm_set_variant(h, variant: int):
    _check(lib().dbm_set_variant(h, int(variant)), "dbm_set_variant")


def dbm_autotune(h, steps: int, stream=None):
    """Returns (best variant, [ms per step of variants 1..8; unused entries 0])."""
    best = ctypes.c_int(0)
    ms = (ctypes.c_float * 8)()
    _check(lib().dbm_autotune(h, int(steps), _stream(stream), ctypes.byref(best), ms), "dbm_autotune")
    return best.value, [ms[i] for i in range(8)]


def dbm_batch_bytes(max_slots: int, max_items: int, precision: int) -> int:
    return int(lib().dbm_batch_bytes(int(max_slots), int(max_items), int(precision)))


def dbm_batch_create(max_slots, max_items, precision, rows_per_item, dev_ptr, nbytes):
    b = ctypes.c_void_p()
    _check(lib().dbm_batch_create(int(max_slots), int(max_items), int(precision), int(rows_per_item),
                                  ctypes.c_void_p(dev_ptr), ctypes.c_size_t(nbytes), ctypes.byref(b)),
           "dbm_batch_create")
    return b


def dbm_batch_destroy(b):
    _check(lib().dbm_batch_destroy(b), "dbm_batch_destroy")


def dbm_batch_attach(b, slot, h, nsteps):
    _check(lib().dbm_batch_attach(b, int(slot), h, int(nsteps)), "dbm_batch_attach")


def dbm_batch_detach(b, slot):
    _check(lib().dbm_batch_detach(b, int(slot)), "dbm_batch_detach")


def dbm_batch_remaining(b, slot) -> int:
    return int(lib().dbm_batch_remaining(b, int(slot)))


def dbm_batch_time(b) -> int:
    return int(lib().dbm_batch_time(b))


def dbm_batch_commit(b, stream=None):
    _check(lib().dbm_batch_commit(b, _stream(stream)), "dbm_batch_commit")


def dbm_batch_step(b, nsteps, stream=None):
    _check(lib().dbm_batch_step(b, int(nsteps), _stream(stream)), "dbm_batch_step")


def dbm_batch_autotune(b, steps: int, stream=None):
    """Returns (variant, rows_per_item, {(variant, rows): ms per step})."""
    v, r = ctypes.c_int(0), ctypes.c_int(0)
    ms = (ctypes.c_float * 8)()
    _check(lib().dbm_batch_autotune(b, int(steps), _stream(stream), ctypes.byref(v), ctypes.byref(r), ms),
           "dbm_batch_autotune")
    return v.value, r.value, list(ms)


def dbm_batch_launch_info(b) -> dict:
    vals = [ctypes.c_int(0) for _ in range(4)]
    _check(lib().dbm_batch_launch_info(b, *[ctypes.byref(v) for v in vals]), "dbm_batch_launch_info")
    return dict(zip(("grid", "items", "rows_per_item", "variant"), [v.value for v in vals]))


# ---- convenience ----------------------------------------------------------

_PREC = {"fp32": DBM_FP32, "fp64": DBM_FP64, DBM_FP32: DBM_FP32, DBM_FP64: DBM_FP64}
_RE = {"explicit": DBM_R_EXPLICIT, "consistent": DBM_R_CONSISTENT, 0: 0, 1: 1}


def params_from(d: dict) -> DbmParams:
    """DbmParams from a dict of paper-named parameters (see workloads.py)."""
    p = dbm_params_default()
    p.nr, p.ntheta = int(d["nr"]), int(d["ntheta"])
    for key in ("r_in", "r_out", "dt", "tau", "Q", "omega1", "omega2", "m", "n", "T_th"):
        if key in d:
            setattr(p, key, float(d[key]))
    if "v" in d:
        for i, val in enumerate(d["v"]):
            p.v[i] = float(val)
    p.precision = _PREC[d.get("precision", "fp32")]
    p.reaction_energy = _RE[d.get("reaction_energy", 0)]
    p.rows_per_item = int(d.get("rows_per_item", 0))
    p.variant = int(d.get("variant", 0))
    p.sector = int(d.get("sector", 0))
    p.r_bc_inner = {"outflow": DBM_BC_OUTFLOW, "centre": DBM_BC_CENTRE, 0: 0, 1: 1}[d.get("r_bc_inner", 0)]
    return p


FIELDS = ("rho", "ur", "uth", "T", "lam")


def _finish_device(buf):
    """Wait for all work on the device that holds buf (every stream)."""
    import torch
    if buf is not None and buf.is_cuda:
        torch.cuda.synchronize(buf.device)


class Simulation:
    """One simulation on the current CUDA device; device memory is a torch
    uint8 tensor that the library borrows for the handle's lifetime."""

    def __init__(self, params, device=None):
        import torch
        self.p = params if isinstance(params, DbmParams) else params_from(params)
        self.nbytes = dbm_state_bytes(self.p)
        if self.nbytes == 0:
            raise DbmError(DBM_EINVAL, "dbm_state_bytes")
        dev = torch.device("cuda" if device is None else device)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.buf.data_ptr()
        self.ptr = (base + 255) // 256 * 256
        self.h = dbm_create(self.p, self.ptr, self.nbytes)

    @property
    def shape(self):
        return (self.p.ntheta, self.p.nr)

    def init_state(self, fields: dict, stream=None):
        dbm_init_state(self.h, *_field_arrays(fields, self.p.nr * self.p.ntheta), stream=stream)

    def step(self, nsteps: int, stream=None):
        dbm_step(self.h, nsteps, stream)

    def moments(self, stream=None, totals=False, raise_nonfinite=True):
        out = {k: np.empty(self.shape) for k in FIELDS}
        tot = np.zeros(4) if totals else None
        st = dbm_moments(self.h, *[out[k] for k in FIELDS], totals=tot, stream=stream,
                         raise_nonfinite=raise_nonfinite)
        if totals:
            out["totals"] = tot
        out["status"] = st
        return out

    def launch_info(self) -> dict:
        return dbm_launch_info(self.h)

    def state_device(self):
        """(f address, lambda address, ld) of the current state on the device."""
        return dbm_state_device(self.h)

    def noneq(self, stream=None):
        """Delta*_m of Sec. II.E: array (12, ntheta, nr), components in NONEQ order."""
        out = np.empty((12,) + self.shape)
        dbm_noneq(self.h, out, stream)
        return out

    def set_variant(self, variant: int):
        dbm_set_variant(self.h, variant)

    def autotune(self, steps: int = 20, stream=None):
        best, ms = dbm_autotune(self.h, steps, stream)
        return best, ms[:dbm_num_variants(self.p.precision)]

    def export_state(self, stream=None):
        dt = np.float64 if self.p.precision == DBM_FP64 else np.float32
        f = np.empty((NV, self.p.ntheta, self.p.nr), dtype=dt)
        lam = np.empty((self.p.ntheta, self.p.nr), dtype=dt)
        steps = dbm_export_state(self.h, f, lam, stream)
        return f, lam, steps

    def import_state(self, f, lam, steps, stream=None):
        dt = np.float64 if self.p.precision == DBM_FP64 else np.float32
        f = np.ascontiguousarray(f, dtype=dt)
        lam = np.ascontiguousarray(lam, dtype=dt)
        n = self.p.nr * self.p.ntheta
        if f.size != NV * n or lam.size != n:
            raise ValueError(f"state of {f.size} + {lam.size} values for {NV} x {n} + {n}")
        dbm_import_state(self.h, f, lam, steps, stream)

    def close(self):
        if self.h is not None:
            # dbm_destroy waits for the work enqueued on the handle's buffers;
            # work the caller queued behind it on the same streams (a copy out
            # of the state, say) is finished too before torch may hand the
            # buffer to another tensor
            _finish_device(self.buf)
            dbm_destroy(self.h)
            self.h = None
            self.buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A batch of simulations advanced together (device tables in a torch
    buffer borrowed by the library)."""

    def __init__(self, max_slots: int, max_items: int, precision="fp32", rows_per_item=0,
                 device=None):
        import torch
        self.precision = _PREC[precision]
        self.nbytes = dbm_batch_bytes(max_slots, max_items, self.precision)
        if self.nbytes == 0:
            raise DbmError(DBM_EINVAL, "dbm_batch_bytes")
        dev = torch.device("cuda" if device is None else device)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=dev)
        self.ptr = (self.buf.data_ptr() + 255) // 256 * 256
        self.b = dbm_batch_create(max_slots, max_items, self.precision, rows_per_item, self.ptr,
                                  self.nbytes)
        self.sims = {}

    def attach(self, slot: int, sim: "Simulation", nsteps: int):
        dbm_batch_attach(self.b, slot, sim.h, nsteps)
        self.sims[slot] = sim

    def detach(self, slot: int):
        dbm_batch_detach(self.b, slot)
        self.sims.pop(slot, None)

    def remaining(self, slot: int) -> int:
        return dbm_batch_remaining(self.b, slot)

    def time(self) -> int:
        return dbm_batch_time(self.b)

    def step(self, nsteps: int, stream=None):
        dbm_batch_step(self.b, nsteps, stream)

    def launch_info(self) -> dict:
        return dbm_batch_launch_info(self.b)

    def autotune(self, steps: int = 64, stream=None):
        return dbm_batch_autotune(self.b, steps, stream)

    def close(self):
        if self.b is not None:
            _finish_device(self.buf)  # queued batched steps read the tables in buf
            dbm_batch_destroy(self.b)
            self.b = None
            self.buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving -------------------------------------------------------------

class DbmServerConfig(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("max_queue", ctypes.c_int32),
                ("quantum", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("max_items", ctypes.c_int64), ("rows_per_item", ctypes.c_int32),
                ("max_bypass", ctypes.c_int32)]


class DbmFields(ctypes.Structure):
    _fields_ = [(k, _dp) for k in FIELDS]


class DbmResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("nr", ctypes.c_int32), ("ntheta", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("steps", ctypes.c_int64)] + \
               [(k, _dp) for k in FIELDS] + \
               [("totals", ctypes.c_double * 4), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_end", ctypes.c_double)]


class DbmServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("submitted", "completed", "failed", "cancelled",
                                                "queued", "running", "updates", "executed",
                                                "pool_free_largest", "batch_time")] + \
               [("status", ctypes.c_int32), ("pad", ctypes.c_int32)]


def _server_lib():
    L = lib()
    if not getattr(L, "_server_ready", False):
        vp = ctypes.c_void_p
        L.dbm_server_min_bytes.argtypes = [ctypes.POINTER(DbmServerConfig)]
        L.dbm_server_min_bytes.restype = ctypes.c_size_t
        L.dbm_server_create.argtypes = [ctypes.POINTER(DbmServerConfig), vp, ctypes.c_size_t,
                                        ctypes.POINTER(vp)]
        L.dbm_submit.argtypes = [vp, ctypes.POINTER(DbmParams), ctypes.POINTER(DbmFields),
                                 ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
        L.dbm_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(DbmResult), ctypes.c_int64]
        L.dbm_result_free.argtypes = [ctypes.POINTER(DbmResult)]
        L.dbm_cancel.argtypes = [vp, ctypes.c_uint64]
        L.dbm_server_stats_get.argtypes = [vp, ctypes.POINTER(DbmServerStats)]
        L.dbm_server_destroy.argtypes = [vp]
        L._server_ready = True
    return L


def dbm_server_min_bytes(cfg: DbmServerConfig) -> int:
    return int(_server_lib().dbm_server_min_bytes(ctypes.byref(cfg)))


def dbm_server_create(cfg: DbmServerConfig, dev_ptr: int, nbytes: int):
    s = ctypes.c_void_p()
    _check(_server_lib().dbm_server_create(ctypes.byref(cfg), ctypes.c_void_p(dev_ptr),
                                           ctypes.c_size_t(nbytes), ctypes.byref(s)),
           "dbm_server_create")
    return s


def dbm_submit(s, params: DbmParams, fields: dict, nsteps: int) -> int:
    arrs = _field_arrays(fields, int(params.nr) * int(params.ntheta))
    f = DbmFields(*[_ptr(a) for a in arrs])
    t = ctypes.c_uint64(0)
    _check(_server_lib().dbm_submit(s, ctypes.byref(params), ctypes.byref(f), int(nsteps),
                                    ctypes.byref(t)), "dbm_submit")
    return t.value


def dbm_poll(s, ticket: int, timeout_us: int = -1):
    """(status, result dict or None); the result's arrays are copied and freed."""
    r = DbmResult()
    st = _server_lib().dbm_poll(s, ctypes.c_uint64(ticket), ctypes.byref(r), int(timeout_us))
    if st != DBM_OK:
        return st, None
    out = {"status": r.status, "steps": r.steps, "totals": np.array(r.totals[:]),
           "t_submit": r.t_submit, "t_start": r.t_start, "t_end": r.t_end}
    n = r.nr * r.ntheta
    for k in FIELDS:
        ptr = getattr(r, k)
        out[k] = (np.ctypeslib.as_array(ptr, shape=(n,)).reshape(r.ntheta, r.nr).copy()
                  if ptr else None)
    _server_lib().dbm_result_free(ctypes.byref(r))
    return st, out


def dbm_cancel(s, ticket: int):
    _check(_server_lib().dbm_cancel(s, ctypes.c_uint64(ticket)), "dbm_cancel")


def dbm_server_stats_get(s) -> dict:
    st = DbmServerStats()
    _check(_server_lib().dbm_server_stats_get(s, ctypes.byref(st)), "dbm_server_stats_get")
    return {k: getattr(st, k) for k, _ in DbmServerStats._fields_ if k != "pad"}


def dbm_server_destroy(s):
    _check(_server_lib().dbm_server_destroy(s), "dbm_server_destroy")


class Server:
    """A serving loop on a torch device pool borrowed by the library."""

    def __init__(self, pool_bytes: int, max_slots=16, max_queue=1024, quantum=64,
                 precision="fp32", max_items=1 << 16, rows_per_item=16, max_bypass=8, device=None):
        import torch
        self.cfg = DbmServerConfig(max_slots, max_queue, quantum, _PREC[precision], max_items,
                                   rows_per_item, max_bypass)
        dev = torch.device("cuda" if device is None else device)
        self.buf = torch.empty(int(pool_bytes) + 256, dtype=torch.uint8, device=dev)
        self.ptr = (self.buf.data_ptr() + 255) // 256 * 256
        self.s = dbm_server_create(self.cfg, self.ptr, int(pool_bytes))

    def submit(self, params, fields, nsteps) -> int:
        p = params if isinstance(params, DbmParams) else params_from(params)
        return dbm_submit(self.s, p, fields, nsteps)

    def poll(self, ticket, timeout_us=-1):
        return dbm_poll(self.s, ticket, timeout_us)

    def cancel(self, ticket):
        dbm_cancel(self.s, ticket)

    def stats(self) -> dict:
        return dbm_server_stats_get(self.s)

    def close(self):
        if self.s is not None:
            dbm_server_destroy(self.s)
            self.s = None
            self.buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
