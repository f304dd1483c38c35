"""Compile the FP64 CPU oracle (plain C + OpenMP) into oracle/liboracle.so.

The oracle is test infrastructure: the CUDA library never links it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mlsd_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force=False, wait=True):
    """Start (and by default finish) the oracle build; returns the Popen if wait=False."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return None
    # -ffp-contract=off keeps x86 and Arm results identical (no fused multiply-add)
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", LIB + ".tmp", SRC, "-lm"]
    p = subprocess.Popen(cmd)
    if not wait:
        return p
    finish(p)
    return None


def finish(p):
    if p is None:
        return
    if p.wait() != 0:
        raise RuntimeError("oracle build failed")
    os.replace(LIB + ".tmp", LIB)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(LIB)
