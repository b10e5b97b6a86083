"""Compile the C oracle into oracle/_build/liboracle.so (test infrastructure).

The flags keep every floating-point operation as written (no contraction into
fused multiply-adds, no fast-math), so the oracle gives the same bits on x86-64
and on aarch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ellsolve_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    deps = [SRC, os.path.join(HERE, "ellsolve_oracle.h")]
    if not force and os.path.exists(LIB):
        if all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in deps):
            return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
