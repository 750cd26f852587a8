"""Builds the oracle shared library (plain C, FP64, no FMA contraction): the
CCZ4 method and the Bowen-York initial-data solve.

Test infrastructure: the library is the independent CPU check of the CUDA
path and is never loaded by the product code.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("ccz4_oracle.c", "bowen_york.c")]
HDRS = [os.path.join(HERE, f) for f in ("ccz4_oracle.h", "bowen_york.h")]
LIB = os.path.join(HERE, "liboracle_ccz4.so")


def build(force: bool = False) -> str:
    """Compiles the oracle if the library is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in SRCS + HDRS)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
           "-Wall", "-Wextra"] + SRCS + ["-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
