"""Build step of the CUDA library ``libledds.so`` (sm_103a only).

Each ``csrc/*.cu`` file is compiled by nvcc in parallel, then linked into
``paper_2512_04997_gb300/_build/libledds.so`` with the CUDA runtime linked statically.
``dem.cu`` is compiled with ``-fmad=false`` so that its FP64 expressions (contact
predicate, cell keys, integrator) round exactly in the order they are written.
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libledds.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
          "--expt-relaxed-constexpr"]
SOURCES = {"lbm.cu": [], "psm_aa.cu": [], "psm_wide.cu": [], "dem.cu": ["-fmad=false"], "api.cu": [],
           "noalloc.cu": ["-fmad=false"]}


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "ledds.h"))
    files.append(os.path.abspath(__file__))
    return files


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile and link the library if it is missing or older than its sources."""
    os.makedirs(OUT, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _inputs())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    nvcc = _nvcc()

    def compile_one(name):
        src = os.path.join(CSRC, name)
        obj = os.path.join(OUT, name.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *COMMON, *SOURCES[name], *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, extra=sys.argv[1:]))
