"""Build libsweep.so (the CUDA library behind include/sweep.h) for sm_103a.

``python -m paper_2105_10332_b300.build`` or ``build()``.  The library is
compiled in-tree, next to this file, with nvcc; no CPU fallback exists.
"""
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsweep.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

# -fmad=false: no implicit contraction; the kernels place every fma explicitly.
# IEEE division and square root are nvcc's defaults (-prec-div, -prec-sqrt).
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-shared", "-I", os.path.join(ROOT, "include")]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "sweep.h")]


# The checked build: kernels also verify their launch geometry and shared
# memory at entry and report a mismatch in the device error word.
LIB_CHECKED = os.path.join(HERE, "libsweep_checked.so")


def build(force=False, verbose=False):
    """Compile libsweep.so and libsweep_checked.so if missing or stale (both
    at once); return the path of libsweep.so."""
    newest = max(os.path.getmtime(f) for f in deps())
    todo = [(path, extra) for path, extra in ((LIB, []), (LIB_CHECKED, ["-DSWEEP_CHECKED"]))
            if force or not os.path.exists(path) or os.path.getmtime(path) < newest]
    procs = []
    for path, extra in todo:
        tmp = path + ".tmp%d" % os.getpid()
        cmd = [NVCC, *FLAGS, *extra, *(["-Xptxas", "-v"] if verbose else []), "-o", tmp, *sources()]
        procs.append((subprocess.Popen(cmd), tmp, path))
    failed = [p.wait() for p, _, _ in procs]
    if any(failed):
        raise subprocess.CalledProcessError(max(failed), NVCC)
    for _, tmp, path in procs:
        os.replace(tmp, path)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
