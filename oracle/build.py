"""Builds the FP64 CPU oracle (test infrastructure) into oracle/libkb_oracle.so.

Plain gcc, OpenMP over start pixels, -ffp-contract=off so that no multiply-add is fused:
the three FP32 operations of the integer track rounding must be the IEEE single operations
the definition names.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kb_oracle.c")
LIB = os.path.join(HERE, "libkb_oracle.so")


def command(src: str = SRC, out: str = LIB) -> list:
    """The gcc command line that builds the oracle source ``src`` into the library ``out``."""
    return ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", "-o", out, src, "-lm"]


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    subprocess.check_call(command())
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
