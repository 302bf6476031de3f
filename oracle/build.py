"""Build the C oracle into oracle/_build/libgf2x_oracle.so (plain gcc).

TEST INFRASTRUCTURE ONLY: the product path never loads this library.
"""
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "gf2x_oracle.c")
LIB = os.path.join(BUILD, "libgf2x_oracle.so")


def build(force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    # The PMULL form of clmul64 exists only for aarch64 compilers; OpenMP is
    # optional.  Each variant is tried in turn, the plainest last.
    pmull = ["-DGF2O_PMULL"] if platform.machine().lower() in ("aarch64", "arm64") else []
    variants = [pmull + ["-fopenmp"], ["-fopenmp"], []]
    if not pmull:
        variants = variants[1:]
    err = ""
    for extra in variants:
        cmd = ["gcc", "-O2", "-fPIC", "-shared"] + extra + ["-o", tmp, SRC]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            break
        err = r.stderr
    else:
        raise RuntimeError("oracle build failed:\n" + err)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
