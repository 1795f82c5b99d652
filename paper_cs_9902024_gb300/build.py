"""In-tree build of libdsmc.so for sm_103a with nvcc (no cmake).

The translation units compile in parallel; the shared library links the
CUDA runtime dynamically (same soname as the one PyTorch loads) with an rpath
to the toolkit.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libdsmc.so")
# (source, object, extra flags): the kernels twice -- FP32 state with fused
# multiply-add contraction, FP64 state without it (rounded as the FP64
# oracle rounds) -- and the host engine
UNITS = [("dsmc_kernels.cu", "dsmc_kernels_f32.o", ["-fmad=true"]),
         ("dsmc_kernels.cu", "dsmc_kernels_f64.o", ["-fmad=false", "-DDSMC_KERNELS_FP64"]),
         ("dsmc_engine.cu", "dsmc_engine.o", ["-fmad=false"])]
HEADERS = [os.path.join(CSRC, "dsmc_internal.cuh"), os.path.join(ROOT, "include", "dsmc.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-O2", "-Xcompiler", "-ffp-contract=off", "-I" + os.path.join(ROOT, "include")]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    return "/usr/local/cuda"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile and link libdsmc.so; returns its path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    objs, procs = [], []
    for src, obj_name, extra in UNITS:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD_DIR, obj_name)
        objs.append(obj)
        if force or _stale(obj, [path] + HEADERS + [os.path.abspath(__file__)]):
            cmd = [nvcc] + NVCC_FLAGS + extra + ["-c", path, "-o", obj + ".tmp"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((subprocess.Popen(cmd), obj))
    for p, obj in procs:
        if p.wait() != 0:
            raise RuntimeError("nvcc failed for %s" % obj)
        os.replace(obj + ".tmp", obj)
    if force or procs or _stale(LIB_PATH, objs):
        tmp = LIB_PATH + ".tmp%d" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
            "-Xlinker", "-rpath", "-Xlinker", os.path.join(cuda, "lib64")]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
