"""Build the CPU oracle shared library (test infrastructure only).

``python oracle/build.py`` compiles ``mf_oracle.c`` into ``oracle/liboracle.so``
with gcc.  Floating-point contraction is disabled so that every fused
multiply-add in the oracle is the explicit ``fma``/``fmaf`` written in the
source.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mf_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "mf_oracle.h"))
    ):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [
        "gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
        "-ffp-contract=off", "-fno-fast-math", "-fno-math-errno",
        SRC, "-o", tmp, "-lm",
    ]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
