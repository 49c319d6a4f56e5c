"""Compile the C oracle into a shared library next to its source.

Test infrastructure: the oracle is the FP64 CPU reference the CUDA path is
checked against. Building it does not make anything use it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liblbm_oracle.so")


def build(force: bool = False) -> str:
    """Build liblbm_oracle.so if missing or older than its source; return its path.

    -ffp-contract=off keeps every multiply and add a separately rounded FP64
    operation, so the oracle's arithmetic is exactly what the C source says.
    """
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
