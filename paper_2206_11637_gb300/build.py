"""Build libpflbm.so in-tree with nvcc for sm_103a (GB300)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpflbm.so")
SOURCES = ["pflbm.cu", "noalloc.cu", "batch.cu"]
DEPS = SOURCES + ["kernels.cuh", "lattice.cuh", "step.cuh", "adjoint.cuh", "errors.h", "host_common.h"]
HEADER = os.path.join(os.path.dirname(HERE), "include", "pflbm.h")

NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
              "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(CSRC, f)) > t for f in DEPS) or os.path.getmtime(HEADER) > t


def build_library(force=False, verbose=False, extra=()):
    """Compile the translation units in parallel, then link the shared library."""
    if not force and not stale():
        return LIB
    tag = ".%d" % os.getpid()
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(CSRC, src[:-3] + tag + ".o")
        cmd = [_nvcc()] + NVCC_FLAGS + list(extra) + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((subprocess.Popen(cmd), cmd))
        objs.append(obj)
    failed = [cmd for pr, cmd in procs if pr.wait() != 0]
    try:
        if failed:
            raise subprocess.CalledProcessError(1, failed[0])
        tmp = LIB + ".tmp" + tag
        cmd = [_nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a"] + objs + ["-o", tmp]
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    build_library(force=True, verbose=True)
