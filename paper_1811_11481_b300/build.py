"""Build libtpc.so in-tree with nvcc for sm_103a (B300).

The finder, merger and compression units are compiled with -fmad=false: their decisions are
taken on single-precision values with one rounding per written operation.
The refit unit (checked against the FP64 oracle within a tolerance) is
compiled with --use_fast_math: fused multiply-adds and approximate
single-precision division and square root.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libtpc.so")
BUILD = os.path.join(ROOT, "_build")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC,
          "--expt-relaxed-constexpr"]
UNITS = {
    "tpc_find.cu": ["-fmad=false"],
    "tpc_refit.cu": ["--use_fast_math"],
    "tpc_capi.cu": [],
    "tpc_noalloc.cu": ["--use_fast_math"],
    "tpc_merge.cu": ["-fmad=false"],
    "tpc_compress.cu": ["-fmad=false"],
}


def sources():
    return [os.path.join(CSRC, f) for f in UNITS] + [
        os.path.join(CSRC, "tpc_math.cuh"), os.path.join(CSRC, "tpc_impl.h"),
        os.path.join(CSRC, "tpc_refit_core.cuh"),
        os.path.join(INC, "tpc.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force=False, verbose=False, extra=()):
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    objs = []
    for unit, flags in UNITS.items():
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        cmd = [NVCC, *ARCH, *COMMON, *flags, *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        objs.append(obj)
    cmd = [NVCC, *ARCH, "-shared", "-o", LIB, *objs]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ("-Xptxas", "-v") if "--ptxas" in sys.argv else ()
    build(force=True, verbose=v, extra=extra)
    print(LIB)
