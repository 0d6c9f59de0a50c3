"""Compile the C part of the oracle (plain gcc, no vendor code).

The oracle is test infrastructure: only the tests, the smoke check and the
benchmark's CPU-baseline leg load it.  Build flags keep every floating-point
operation separately rounded (no contraction into fused multiply-adds), so
the oracle evaluates each formula exactly as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libpic_oracle.so")
SRC = [os.path.join(HERE, "pic_oracle.c")]


def _stale():
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    return any(os.path.getmtime(s) > t for s in SRC)


def build(force=False, openmp=False):
    """Build libpic_oracle.so into oracle/_build; returns its path."""
    if not force and not _stale():
        return SO
    os.makedirs(BUILD, exist_ok=True)
    tmp = SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + SRC + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
