"""Compile oracle/oracle.c into oracle/_build/liboracle.so with the host C compiler.

Test infrastructure only (see oracle/oracle.c).  x86-64 uses libquadmath's
__float128; AArch64 uses its native binary128 ``long double``.
"""
import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    # no contraction of products into FMAs: the error-free transformations of oracle.c
    # (two-sum, FMA residuals) need every other operation rounded as written
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", SRC, "-o", LIB + ".tmp",
           "-lm"]
    if platform.machine() not in ("aarch64", "arm64"):
        cmd.append("-lquadmath")
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
