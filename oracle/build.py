"""Compile the CPU oracle (test infrastructure) into oracle/_build/libngb_oracle.so.

Plain g++ (C++17, portable, no target-specific flags) with -ffp-contract=off so
that FP32 expressions are evaluated operation by operation, as written.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ngb_oracle.cpp")
HDR = os.path.join(HERE, "ngb_oracle.h")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libngb_oracle.so")


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its sources; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
           "-Wall", "-Wextra", "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
