"""Builds the CPU oracle (plain C, FP64, OpenMP) into oracle/_build/.

Test infrastructure only: the library's product path never builds, loads or
calls it.  Flags keep IEEE double semantics on every host: no fast-math and
no contraction of a*b+c into fused multiply-adds.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ptdr_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libptdr_oracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = [
        os.environ.get("CC", "gcc"), "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared",
        "-ffp-contract=off", "-fno-fast-math", SRC, "-o", LIB + ".tmp", "-lm",
    ]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
