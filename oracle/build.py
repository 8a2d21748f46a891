"""Build the C oracle (2D and 3D) into oracle/libstokes_oracle.so (plain gcc, FP64).

Test infrastructure only: the oracle is loaded by the tests, the smoke check
and the CPU-baseline leg of the benchmark, never by the product path.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "stokes_oracle.c")
SRCS = [SRC, os.path.join(HERE, "stokes3d_oracle.c")]
LIB = os.path.join(HERE, "libstokes_oracle.so")

# -ffp-contract=off: every product and sum is rounded exactly where it is written.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall", "-Wextra"]


LIB_OMP = os.path.join(HERE, "libstokes_oracle_omp.so")


def build_oracle_omp(force: bool = False) -> str:
    """The same sources built with OpenMP (the RAS tiles of one outer
    iteration run in parallel); used only for the all-cores CPU baseline."""
    if force or not os.path.exists(LIB_OMP) or os.path.getmtime(LIB_OMP) < max(os.path.getmtime(s) for s in SRCS):
        tmp = LIB_OMP + ".tmp.%d" % os.getpid()
        subprocess.run(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, *SRCS, "-lm"], check=True)
        os.replace(tmp, LIB_OMP)
    return LIB_OMP


def build_oracle(force: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(s) for s in SRCS):
        tmp = LIB + ".tmp.%d" % os.getpid()
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, *SRCS, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
