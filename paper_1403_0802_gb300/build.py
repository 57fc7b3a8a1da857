"""Build libsj.so in-tree with nvcc for sm_103a (GB300).

Each .cu file is compiled in parallel to an object file, then nvcc links the
shared library (CUDA runtime linked statically).  Outputs go to
paper_1403_0802_gb300/_build/ (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
SO = os.path.join(OUT, "libsj.so")
SOURCES = ["sj_api.cu", "sj_engine.cu", "sj_filter.cu", "sj_pip.cu", "sj_p2p.cu", "sj_peaks.cu", "sj_serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    inc = os.path.join(ROOT, "include")
    return ([os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(inc, f) for f in os.listdir(inc)]
            + [os.path.abspath(__file__)])


SO_CHECKED = os.path.join(OUT, "checked", "libsj.so")   # bounds-checked build (SJ_CHECK_BOUNDS)


def up_to_date(so: str = SO) -> bool:
    if not os.path.exists(so):
        return False
    t = os.path.getmtime(so)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Compile libsj.so (checked=True: the bounds-checked build, in
    _build/checked/, with -DSJ_CHECK_BOUNDS) and return its path."""
    so = SO_CHECKED if checked else SO
    out = os.path.dirname(so)
    if checked:
        extra = (*extra, "-DSJ_CHECK_BOUNDS")
    if not force and up_to_date(so):
        return so
    os.makedirs(out, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(out, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = so + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else []))
