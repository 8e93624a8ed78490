"""Compile the CUDA library ``libfloodped.so`` for sm_103a (B300), in-tree.

Each translation unit is compiled separately, all with -fmad=false: every
fused multiply-add in the kernels is written out explicitly, so a device
function gives the same bits in every kernel it is inlined into.  The CUDA
runtime is linked statically.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libfloodped.so")
OBJ = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC]
SOURCES = [("flood.cu", []), ("peds.cu", []), ("floodped.cu", []), ("noalloc.cu", []), ("persist.cu", []), ("surrogate.cu", []), ("window.cu", []), ("muscl.cu", []), ("batch.cu", [])]


def _inputs():
    out = [os.path.join(INC, "floodped.h")]
    for f in os.listdir(CSRC):
        out.append(os.path.join(CSRC, f))
    return out


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    objs = []
    for src, flags in SOURCES:
        obj = os.path.join(OBJ, src.replace(".cu", ".o"))
        cmd = ["nvcc"] + ARCH + COMMON + flags + (["-Xptxas", "-v"] if verbose else []) + [
            "-c", os.path.join(CSRC, src), "-o", obj]
        subprocess.check_call(cmd)
        objs.append(obj)
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["nvcc"] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
