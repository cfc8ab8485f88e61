"""Build step of the FP64 CPU oracle (test infrastructure only).

Compiles ``ledds_oracle.c`` with gcc into ``oracle/_build/libledds_oracle.so``: no
floating-point contraction, no fast-math, no host-specific instruction set, so the x86
container and the Arm GPU host give identical results. The parity tests use this build.

``build(parallel=True)`` compiles the same source a second time with OpenMP
(``libledds_oracle_omp.so``, -O3 -fopenmp, the same IEEE flags): the lattice update runs
on every host core. It is the timed CPU baseline of the benchmark and is used for nothing
else (its per-particle force sums are added in a varying order).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libledds_oracle.so")
LIB_OMP = os.path.join(OUT_DIR, "libledds_oracle_omp.so")
SRC = os.path.join(HERE, "ledds_oracle.c")
HDR = os.path.join(HERE, "ledds_oracle.h")


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile the oracle if its shared library is missing or older than its sources."""
    os.makedirs(OUT_DIR, exist_ok=True)
    out = LIB_OMP if parallel else LIB
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR), os.path.getmtime(__file__))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    tmp = out + f".tmp{os.getpid()}"
    opt = ["-O3", "-fopenmp"] if parallel else ["-O2"]
    cmd = ["gcc", *opt, "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-Wno-unknown-pragmas", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
    print(build(force=True, parallel=True))
