"""Build the C part of the oracle (TEST INFRASTRUCTURE ONLY) into oracle/_build/liboracle_sweep.so."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "_build", "liboracle_sweep.so")


def build(force=False):
    src = os.path.join(HERE, "csweep.c")
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(src):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    # -O3 without -march=native: the same source builds on the x86 and Arm hosts with the same results (ISO C99
    # mode keeps floating-point contraction off, so no FMA is formed on either)
    subprocess.check_call(["gcc", "-O3", "-std=c99", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
