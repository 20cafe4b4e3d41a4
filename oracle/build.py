"""Compile the C part of the oracle (test infrastructure only).

The oracle is the slow FP64 reference that tests and the CPU-baseline leg of
the benchmark use; nothing in the CUDA library links or calls it.

Flags: -O2 with IEEE semantics (no -ffast-math) and -ffp-contract=off so that
x86-64 and aarch64 hosts evaluate the same FP64 expression tree.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "mc_oracle.c")]


def build(force: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in SOURCES)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp] + SOURCES + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
