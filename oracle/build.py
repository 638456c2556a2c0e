"""Compile the CPU oracle (plain C, FP64) into ``oracle/liboracle.so``.

Test infrastructure only: the oracle checks the CUDA library and is never part of it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["or_codec.c", "or_mpm.c", "or_scheme.c", "or_adjoint.c", "or_smoke.c"]
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")


def build(force: bool = False, threaded: bool = False) -> str:
    """The sequential oracle (default), or the OpenMP build of the same sources that only
    long FP64 reference rollouts use (``threaded``)."""
    lib = LIB_OMP if threaded else LIB
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    deps = srcs + [os.path.join(HERE, "oracle.h"), os.path.abspath(__file__)]
    if not force and os.path.exists(lib):
        lib_m = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= lib_m for d in deps):
            return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
           "-Wno-unknown-pragmas"] + (["-fopenmp"] if threaded else []) + ["-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build(force="--force" in sys.argv, threaded=True))
