"""Build ``liblbm_gb300.so`` in-tree with nvcc for sm_103a.

Each lattice's kernels live in their own translation unit; the units are
compiled in parallel and linked into one shared library that exports the C-ABI
of ``include/lbm.h``.  The CUDA runtime is linked shared, so the process shares
one runtime (and therefore streams) with PyTorch.

``build(bounds_check=True)`` builds the bounds-check variant
``liblbm_gb300_bounds.so`` (``-DLBM_DEBUG_BOUNDS``, objects in ``_build_bounds``):
every kernel checks its load and store indices and reports an index outside its
buffer as LBM_ERR_BOUNDS.  ``LBM_BOUNDS_CHECK=1`` makes the binding load it.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm_gb300.so")
BUILD_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB_BOUNDS = os.path.join(HERE, "liblbm_gb300_bounds.so")

UNITS = ["lbm_api.cu", "lbm_inst_d2q9.cu", "lbm_inst_d3q15.cu", "lbm_inst_d3q19.cu", "lbm_inst_d3q27.cu",
         "lbm_inst_d3q39.cu", "lbm_inst_d3q39_k2.cu", "lbm_inst_d3q39_k3.cu", "lbm_inst_d3q39_k4.cu",
         "lbm_inst_d3q39_k5.cu", "lbm_batch.cu", "lbm_noalloc.cu", "lbm_bounds.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _sources():
    return [os.path.join(CSRC, u) for u in UNITS if os.path.exists(os.path.join(CSRC, u))]


def _headers():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
        os.path.join(ROOT, "include", "lbm.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None, bounds_check: bool = False) -> str:
    build_dir, lib = (BUILD_BOUNDS, LIB_BOUNDS) if bounds_check else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    srcs = _sources()
    hdrs = _headers()
    flags = FLAGS + (["-DLBM_DEBUG_BOUNDS"] if bounds_check else []) + list(extra_flags or [])

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        if force or _stale(obj, [src] + hdrs):
            cmd = [nvcc] + ARCH + flags + ["-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
            if verbose and r.stderr.strip():
                print(r.stderr)
        return obj

    order = sorted(srcs, key=lambda f: 0 if "d3q39_k" in f else 1)  # longest units start first
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        done = dict(zip(order, ex.map(compile_one, order)))
    objs = [done[f] for f in srcs]
    if force or _stale(lib, objs):
        tmp = lib + ".tmp.%d" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
            "-ldl", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]  # -ldl: the NVTX loader (lbm_trace.h)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds_check="--bounds" in sys.argv))
