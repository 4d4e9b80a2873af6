"""Compile the plain-C FP64 oracle (test infrastructure) into
oracle/liboracle.so (single thread, the reference form) and, from the same
source with -fopenmp, oracle/liboracle_omp.so (the multi-core leg of the
CPU baseline; its parallel loops give results identical to the first)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gfors_oracle.c")
OUT = os.path.join(HERE, "liboracle.so")
OUT_OMP = os.path.join(HERE, "liboracle_omp.so")


def build(force: bool = False, omp: bool = False) -> str:
    out = OUT_OMP if omp else OUT
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(SRC)):
        return out
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", *(["-fopenmp"] if omp else []), SRC, "-o", out, "-lm"]
    subprocess.check_call(cmd)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build(force="--force" in sys.argv, omp=True))
