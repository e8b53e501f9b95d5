"""Build libgksl.so for sm_103a in-tree (``paper_1812_11626_gb300/_build/``).

Each translation unit is compiled with nvcc in parallel and linked into one shared
library with a plain C ABI (``include/gksl.h``).  No torch headers are involved.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgksl.so")
UNITS = ["prim.cu", "expand.cu", "structure.cu", "assemble.cu", "hyb.cu", "rk4.cu", "adjoint.cu", "batch.cu",
         "api.cu", "noalloc.cu", "mfree.cu", "dense_diss.cu", "rates.cu", "rk4_block.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
         "--expt-relaxed-constexpr"]


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    deps = [src] + [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cuh")]
    deps.append(os.path.join(HERE, "..", "include", "gksl.h"))
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(unit, extra):
    src = os.path.join(SRC, unit)
    obj = os.path.join(OUT, unit.replace(".cu", ".o"))
    if not _stale(obj, src):
        return obj, ""
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, extra=()):
    """Compile every unit (in parallel) and link libgksl.so; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    extra = list(extra)
    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        res = list(ex.map(lambda u: _compile(u, extra), UNITS))
    objs = [o for o, _ in res]
    if verbose:
        for (_, log), u in zip(res, UNITS):
            if log.strip():
                print(f"--- {u}\n{log}", file=sys.stderr)
    if not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
