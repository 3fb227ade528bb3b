"""Build the CUDA library libdbm.so (sm_103a) in-tree.

Each translation unit (FP32 kernels, FP64 kernels, C-ABI runtime) is compiled
by its own nvcc process in parallel, then linked into one shared library with
the CUDA runtime linked statically (no runtime-library path needed).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libdbm.so")
# DBM_DEBUG=1 in the environment: the checked build (device-side bounds and
# alignment checks of every copy and store, see dbm_device.cuh), kept apart
OUT_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(OUT_DEBUG, "libdbm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INC, "-I" + CSRC]
UNITS = ["dbm_fp32.cu", "dbm_fp64.cu", "dbm_api.cu", "dbm_server.cu", "dbm_noalloc.cu"]


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + \
           [os.path.join(INC, f) for f in os.listdir(INC)]


def nvcc():
    for cand in ("nvcc", "/usr/local/cuda/bin/nvcc"):
        try:
            subprocess.run([cand, "--version"], check=True, capture_output=True)
            return cand
        except (OSError, subprocess.CalledProcessError):
            continue
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdbm.so")


def debug_requested() -> bool:
    return os.environ.get("DBM_DEBUG", "") == "1"


def build(force: bool = False, verbose: bool = False, debug: bool | None = None) -> str:
    """Compile libdbm.so if missing or older than any source; returns its path.
    debug (default: DBM_DEBUG=1 in the environment) builds the checked library."""
    if debug is None:
        debug = debug_requested()
    out_dir, lib = (OUT_DEBUG, LIB_DEBUG) if debug else (OUT, LIB)
    flags = FLAGS + (["-DDBM_DEBUG"] if debug else [])
    os.makedirs(out_dir, exist_ok=True)
    if not force and os.path.exists(lib):
        if os.path.getmtime(lib) >= max(os.path.getmtime(p) for p in _sources()):
            return lib
    cc = nvcc()
    procs = []
    objs = []
    for u in UNITS:
        obj = os.path.join(out_dir, u.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc, *ARCH, *flags, "-c", os.path.join(CSRC, u), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for u, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((u, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"--- {u}\n{o}" for u, o in failed))
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-Xlinker", "--exclude-libs,ALL",
           "-Xlinker", "-Bsymbolic", "-o", tmp, *objs]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                debug=True if "--debug" in sys.argv else None))
