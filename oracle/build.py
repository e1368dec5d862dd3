"""Build the FFM oracle shared library (test infrastructure only).

Compiles oracle/ffm_oracle.c and oracle/nufft_oracle.c with gcc into
oracle/libffm_oracle.so.  FP contraction is
off so that every FP64 operation rounds exactly as written; OpenMP parallelises the
outer loops only.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("ffm_oracle.c", "nufft_oracle.c", "nufft_oracle.h")]
LIB = os.path.join(HERE, "libffm_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(f) for f in SRCS):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", "-Wall", "-o", tmp] + [f for f in SRCS if f.endswith(".c")] + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
