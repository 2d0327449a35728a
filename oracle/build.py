"""Compile the FP64 CPU oracle (test infrastructure): oracle/liboracle.so,
one host thread, and oracle/liboracle_omp.so, the same source with OpenMP
over the particle and pair loops (bit for bit the same results).

Plain gcc, no vector intrinsics; -ffp-contract=off so that every
single-precision product and sum in the predicate is rounded on its own.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dem_oracle.c")
OUT = os.path.join(HERE, "liboracle.so")


OUT_OMP = os.path.join(HERE, "liboracle_omp.so")


def build(force: bool = False, parallel: bool = False) -> str:
    """Build (if stale) and return the path of the serial library, or of the
    OpenMP one with parallel=True."""
    out = OUT_OMP if parallel else OUT
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(SRC),
                                             os.path.getmtime(os.path.join(HERE, "dem_oracle.h")),
                                             os.path.getmtime(os.path.abspath(__file__)))):
        return out
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", out + ".tmp", SRC, "-lm"]
    if parallel:
        cmd[1:1] = ["-fopenmp", "-DORC_OPENMP"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build_all(force: bool = False) -> None:
    build(force=force)
    build(force=force, parallel=True)


if __name__ == "__main__":
    build_all(force="--force" in sys.argv)
    print(OUT, OUT_OMP)
