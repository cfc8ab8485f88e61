"""Build step of the FP64 CPU oracle (test infrastructure only).

Compiles ``ledds_oracle.c`` with gcc into ``oracle/_build/libledds_oracle.so``. The flags
keep IEEE semantics: no floating-point contraction, no fast-math, no host-specific
instruction set, so the x86 container and the Arm GPU host give identical results.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libledds_oracle.so")
SRC = os.path.join(HERE, "ledds_oracle.c")
HDR = os.path.join(HERE, "ledds_oracle.h")


def build(force: bool = False) -> str:
    """Compile the oracle if its shared library is missing or older than its sources."""
    os.makedirs(OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
