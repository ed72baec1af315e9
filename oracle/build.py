"""Compile the FP64 CPU oracle (test infrastructure) with gcc.

The oracle is plain C; it is built with IEEE semantics (no fast-math, no
floating-point contraction) so that its results do not depend on whether
the host compiler would fuse multiply-adds (x86 and Arm differ there).
OpenMP is used when the compiler supports it; the arithmetic of every
output is the same with or without it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "onmf_oracle.c")
LIB = os.path.join(HERE, "libonmf_oracle.so")


def build_oracle(force=False):
    """Build libonmf_oracle.so next to its source; return its path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math"]
    tmp = LIB + ".tmp.%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
