"""Compile the oracle's C source into a shared library beside it.

TEST INFRASTRUCTURE (see oracle/__init__.py).  gcc with -O2 -ffp-contract=off,
so no multiply-add is contracted and every expression rounds as written, and
with OpenMP for the cell and edge loops.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "volna_oracle.c")
AD_SRC = os.path.join(HERE, "volna_oracle_ad.cpp")
AD_HDR = os.path.join(HERE, "ad_tape.hpp")
COUNT_SRC = os.path.join(HERE, "volna_oracle_count.cpp")
COUNT_HDR = os.path.join(HERE, "op_count.hpp")


def library_path() -> str:
    return os.path.join(HERE, "_build", "libvolna_oracle.so")


def ad_library_path() -> str:
    return os.path.join(HERE, "_build", "libvolna_oracle_ad.so")


def count_library_path() -> str:
    return os.path.join(HERE, "_build", "libvolna_oracle_count.so")


def build_count(verbose: bool = False) -> str:
    """The oracle compiled with the operation-counting scalar; no OpenMP."""
    out = count_library_path()
    os.makedirs(os.path.dirname(out), exist_ok=True)
    newest = max(os.path.getmtime(f) for f in (SRC, COUNT_SRC, COUNT_HDR))
    if os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c++17",
           "-o", out + ".tmp", COUNT_SRC, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build_ad(verbose: bool = False) -> str:
    """The oracle compiled with the taping scalar (its discrete adjoint); no OpenMP."""
    out = ad_library_path()
    os.makedirs(os.path.dirname(out), exist_ok=True)
    newest = max(os.path.getmtime(f) for f in (SRC, AD_SRC, AD_HDR))
    if os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c++17",
           "-o", out + ".tmp", AD_SRC, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build(verbose: bool = False) -> str:
    out = library_path()
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-Wall", "-o", out + ".tmp", SRC, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build(verbose=True))
    print(build_ad(verbose=True))
    print(build_count(verbose=True))
