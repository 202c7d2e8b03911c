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


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
