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
SO_OMP = os.path.join(BUILD, "libpic_oracle_omp.so")   # the same source with OpenMP (timing only)
SRC = [os.path.join(HERE, "pic_oracle.c")]


def _stale(so):
    if not os.path.exists(so):
        return True
    t = os.path.getmtime(so)
    return any(os.path.getmtime(s) > t for s in SRC)


def build(force=False, openmp=False):
    """Build libpic_oracle.so (or, with openmp, libpic_oracle_omp.so: the
    particle loop shared between threads, for the all-cores CPU baseline) into
    oracle/_build; returns its path."""
    so = SO_OMP if openmp else SO
    if not force and not _stale(so):
        return so
    os.makedirs(BUILD, exist_ok=True)
    tmp = so + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"] + \
          (["-fopenmp"] if openmp else []) + ["-o", tmp] + SRC + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build(force="--force" in sys.argv, openmp=True))
