"""Build libpeps.so in-tree with nvcc for sm_103a (no CMake, parallel units)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libpeps.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def _compile(src: str, obj: str, extra) -> None:
    cmd = [nvcc_path(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
           "--expt-relaxed-constexpr", *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")


def build_library(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile every csrc/*.cu to an object (in parallel) and link libpeps.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = _sources()
    newest_dep = max(os.path.getmtime(p) for p in srcs + _headers())
    objs = [os.path.join(OUT_DIR, os.path.basename(s)[:-3] + ".o") for s in srcs]
    todo = []
    for s, o in zip(srcs, objs):
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), newest_dep):
            todo.append((s, o))
    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(todo)))) as ex:
        futs = [ex.submit(_compile, s, o, list(extra)) for s, o in todo]
        for f in futs:
            f.result()
    if todo or not os.path.exists(LIB):
        cmd = [nvcc_path(), "-shared", *ARCH, "-cudart", "shared", "-o", LIB, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
    if verbose:
        print(f"built {LIB} ({len(todo)} units recompiled)")
    return LIB


if __name__ == "__main__":
    build_library(force=True, verbose=True)
