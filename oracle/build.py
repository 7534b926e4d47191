"""Build the CPU oracle (test infrastructure only) as a shared library.

Plain gcc, -O2, no fast-math, -ffp-contract=off so x86 and Arm hosts produce
identical bits.  OpenMP parallelises over independent domains only.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "grprec_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force=False):
    """Compile liboracle.so next to its source; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "grprec_oracle.h"))):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp",
           "-std=gnu99", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
