"""Build the oracle's shared library (test infrastructure only).

gcc, plain C99, -O2 -ffp-contract=off (every operation rounds as written).
liboracle.so: OpenMP off, so the oracle runs exactly as a reader sees it.
liboracle_omp.so: the same sources with -fopenmp: the loops of a stage that
carry `omp parallel for` run over the host's cores (each cell or face is
computed by the same code, so the results are bit-identical; the only
reductions are a maximum and an error code).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["mhd.c", "eos.c", "mlp.c", "diffusion.c", "poisson.c", "sphere.c"]
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")


def _build_one(lib, extra, srcs, deps, force):
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(s) <= t for s in deps):
            return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"] + extra + \
        ["-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    deps = srcs + [os.path.join(HERE, "oracle.h"), os.path.abspath(__file__)]
    _build_one(LIB, [], srcs, deps, force)
    _build_one(LIB_OMP, ["-fopenmp"], srcs, deps, force)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
