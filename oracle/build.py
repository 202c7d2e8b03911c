"""TEST INFRASTRUCTURE: builds the CPU oracle (plain C, FP64) into oracle/liboracle.so.

Only tests/, the smoke check and the benchmark's CPU-baseline leg use the
result.  -ffp-contract=off keeps gcc from fusing multiply-adds on its own
(aarch64 gcc does so by default), so that x86 and Arm builds round the same.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bicgsafe_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
# The same source built with OpenMP: row loops and inner products over all
# host cores, bit-identical results.  Used only to time the CPU baseline on
# every core; the parity oracle is the single-threaded LIB.
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")


def build(force: bool = False, parallel: bool = False) -> str:
    lib = LIB_OMP if parallel else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"] + \
        (["-fopenmp"] if parallel else []) + ["-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
    print(build(force=True, parallel=True))
