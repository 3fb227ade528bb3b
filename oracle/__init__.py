"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does.

Arrays follow the conventions in ``dbm_oracle.h``: macroscopic fields are
float64 arrays of shape (ntheta, nr); the distribution is (33, ntheta, nr).
"""
import ctypes
import os

import numpy as np

from . import build as _build

NV = 33

_c_double_p = ctypes.POINTER(ctypes.c_double)


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nr", ctypes.c_int),
        ("ntheta", ctypes.c_int),
        ("r_in", ctypes.c_double),
        ("r_out", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("Q", ctypes.c_double),
        ("omega1", ctypes.c_double),
        ("omega2", ctypes.c_double),
        ("m", ctypes.c_double),
        ("n", ctypes.c_double),
        ("T_th", ctypes.c_double),
        ("v", ctypes.c_double * 4),
        ("reaction_energy", ctypes.c_int),
        ("sector", ctypes.c_int),
        ("r_bc_inner", ctypes.c_int),
    ]


DEFAULTS = dict(r_in=0.05, r_out=1.05, dt=1e-5, tau=1e-3, Q=1.0, omega1=0.0,
                omega2=0.0, m=1.0, n=1.0, T_th=1.1, v=(1.5, 3.5, 7.5, 12.5),
                reaction_energy=0, sector=0, r_bc_inner=0)


def make_params(**kw) -> OracleParams:
    """Build the oracle's parameter struct from keyword arguments (paper names)."""
    d = dict(DEFAULTS)
    d.update(kw)
    p = OracleParams()
    p.nr = int(d["nr"])
    p.ntheta = int(d["ntheta"])
    for key in ("r_in", "r_out", "dt", "tau", "Q", "omega1", "omega2", "m", "n", "T_th"):
        setattr(p, key, float(d[key]))
    for i, val in enumerate(d["v"]):
        p.v[i] = float(val)
    re = d["reaction_energy"]
    p.reaction_energy = {"explicit": 0, "consistent": 1}.get(re, re)
    p.sector = int(d["sector"])
    bc = d["r_bc_inner"]
    p.r_bc_inner = {"outflow": 0, "centre": 1}.get(bc, bc)
    return p


_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(OracleParams)
        dp = _c_double_p
        L.oracle_weights.argtypes = [dp, ctypes.c_double, dp]
        L.oracle_velocities.argtypes = [dp, ctypes.c_double, dp, dp]
        L.oracle_feq.argtypes = [dp, ctypes.c_double] + [ctypes.c_double] * 4 + [dp]
        L.oracle_site_moments.argtypes = [dp, ctypes.c_double, dp] + [dp] * 4
        L.oracle_chem.argtypes = [dp, ctypes.c_double] + [ctypes.c_double] * 6 + [dp]
        L.oracle_rate.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
        L.oracle_rate.restype = ctypes.c_double
        L.oracle_lambda_react.argtypes = [ctypes.c_double] * 4
        L.oracle_lambda_react.restype = ctypes.c_double
        L.oracle_init.argtypes = [P] + [dp] * 7
        L.oracle_step.argtypes = [P, dp, dp, dp, dp]
        L.oracle_step.restype = ctypes.c_long
        L.oracle_macro.argtypes = [P, dp, dp] + [dp] * 5
        L.oracle_totals.argtypes = [P, dp, dp]
        L.oracle_run.argtypes = [P] + [dp] * 5 + [ctypes.c_long] + [dp] * 5
        L.oracle_run.restype = ctypes.c_int
        L.oracle_central_moments.argtypes = [dp, ctypes.c_double, dp, ctypes.c_double,
                                             ctypes.c_double, dp]
        L.oracle_noneq.argtypes = [P, dp, dp]
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_set_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "float64 C-contiguous array expected"
    return a.ctypes.data_as(_c_double_p)


def _vec(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64))


def set_threads(n: int) -> int:
    """OpenMP threads for oracle_step (n < 1: all processors)."""
    return lib().oracle_set_threads(int(n))


def weights(T, v=DEFAULTS["v"]):
    F = np.zeros(5)
    lib().oracle_weights(_ptr(_vec(v)), float(T), _ptr(F))
    return F


def velocities(theta, v=DEFAULTS["v"]):
    vr, vth = np.zeros(NV), np.zeros(NV)
    lib().oracle_velocities(_ptr(_vec(v)), float(theta), _ptr(vr), _ptr(vth))
    return vr, vth


def feq(theta, rho, ur, uth, T, v=DEFAULTS["v"]):
    out = np.zeros(NV)
    lib().oracle_feq(_ptr(_vec(v)), float(theta), float(rho), float(ur), float(uth),
                     float(T), _ptr(out))
    return out


def site_moments(theta, f, v=DEFAULTS["v"]):
    f = _vec(f)
    out = [ctypes.c_double() for _ in range(4)]
    lib().oracle_site_moments(_ptr(_vec(v)), float(theta), _ptr(f),
                              *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def chem(theta, rho, ur, uth, T, Q, R, v=DEFAULTS["v"]):
    out = np.zeros(NV)
    lib().oracle_chem(_ptr(_vec(v)), float(theta), float(rho), float(ur), float(uth),
                      float(T), float(Q), float(R), _ptr(out))
    return out


def rate(p, rho, T, lam):
    a, b = ctypes.c_double(), ctypes.c_double()
    R = lib().oracle_rate(ctypes.byref(p), float(rho), float(T), float(lam),
                          ctypes.byref(a), ctypes.byref(b))
    return R, a.value, b.value


def lambda_react(lam, a, b, dt):
    return lib().oracle_lambda_react(float(lam), float(a), float(b), float(dt))


def _fields(p, fields):
    shape = (p.ntheta, p.nr)
    out = []
    for name in ("rho", "ur", "uth", "T", "lam"):
        a = np.ascontiguousarray(np.asarray(fields[name], dtype=np.float64))
        assert a.shape == shape, (name, a.shape, shape)
        out.append(a)
    return out


def init(p, fields):
    """f = f^eq of the macroscopic fields; returns (f, lam)."""
    rho, ur, uth, T, lam = _fields(p, fields)
    N = p.nr * p.ntheta
    f = np.zeros((NV, p.ntheta, p.nr))
    lf = np.zeros((p.ntheta, p.nr))
    lib().oracle_init(ctypes.byref(p), _ptr(rho), _ptr(ur), _ptr(uth), _ptr(T), _ptr(lam),
                      _ptr(f), _ptr(lf))
    assert f.size == NV * N
    return f, lf


def step(p, f, lam):
    """One time step; returns (f_new, lam_new, n_clamped)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    fn = np.empty_like(f)
    ln = np.empty_like(lam)
    c = lib().oracle_step(ctypes.byref(p), _ptr(f), _ptr(lam), _ptr(fn), _ptr(ln))
    return fn, ln, int(c)


def macro(p, f, lam):
    """Macroscopic fields of a state as a dict of (ntheta, nr) arrays."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    out = {k: np.zeros((p.ntheta, p.nr)) for k in ("rho", "ur", "uth", "T", "lam")}
    lib().oracle_macro(ctypes.byref(p), _ptr(f), _ptr(lam), _ptr(out["rho"]), _ptr(out["ur"]),
                       _ptr(out["uth"]), _ptr(out["T"]), _ptr(out["lam"]))
    return out


def totals(p, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    t = np.zeros(4)
    lib().oracle_totals(ctypes.byref(p), _ptr(f), _ptr(t))
    return t


def run(p, fields, nsteps):
    """init + nsteps steps + macro; returns a dict of (ntheta, nr) arrays."""
    rho, ur, uth, T, lam = _fields(p, fields)
    out = {k: np.zeros((p.ntheta, p.nr)) for k in ("rho", "ur", "uth", "T", "lam")}
    rc = lib().oracle_run(ctypes.byref(p), _ptr(rho), _ptr(ur), _ptr(uth), _ptr(T), _ptr(lam),
                          int(nsteps), _ptr(out["rho"]), _ptr(out["ur"]), _ptr(out["uth"]),
                          _ptr(out["T"]), _ptr(out["lam"]))
    if rc != 0:
        raise MemoryError("oracle_run: allocation failed")
    return out


NONEQ = ("d2_rr", "d2_rth", "d2_thth", "d3_rrr", "d3_rrth", "d3_rthth", "d3_ththth",
         "d31_r", "d31_th", "d42_rr", "d42_rth", "d42_thth")


def central_moments(theta, g, ur, uth, v=DEFAULTS["v"]):
    out = np.zeros(12)
    lib().oracle_central_moments(_ptr(_vec(v)), float(theta), _ptr(_vec(g)), float(ur), float(uth),
                                 _ptr(out))
    return out


def noneq(p, f):
    """Delta*_m of Sec. II.E at every site: array (12, ntheta, nr), components in NONEQ order."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros((12, p.ntheta, p.nr))
    lib().oracle_noneq(ctypes.byref(p), _ptr(f), _ptr(out))
    return out
