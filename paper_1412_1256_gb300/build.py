"""Build the CUDA library ``libpolaris.so`` in-tree (sm_103a only).

Every ``csrc/*.cu`` file is compiled to an object in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3``) and the objects are
linked into ``paper_1412_1256_gb300/libpolaris.so``.  Objects live in
``paper_1412_1256_gb300/_build/``; a source is recompiled when it, or a header in
``csrc/`` or ``include/``, is newer than its object.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpolaris.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    for c in ("/usr/local/cuda/bin/nvcc",):
        if os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _newest_header() -> float:
    hs = (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
          glob.glob(os.path.join(ROOT, "include", "*.h")))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, out_dir: str | None = None,
          defines: tuple = ()) -> str:
    """Compile and link libpolaris.so; return its path.  out_dir/defines build a variant
    (objects and library in out_dir, extra -D flags) without touching the default build."""
    BUILD = os.path.join(out_dir, "_build") if out_dir else globals()["BUILD"]
    LIB = os.path.join(out_dir, "libpolaris.so") if out_dir else globals()["LIB"]
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_t = _newest_header()
    todo = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_t):
            todo.append((s, o))

    def comp(so):
        s, o = so
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *[f"-D{d}" for d in defines], "-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(s)}:\n{r.stderr[-4000:]}")
        os.replace(o + ".tmp", o)
        if verbose:
            print("compiled", os.path.basename(s), flush=True)

    if todo:
        jobs = jobs or min(len(todo), max(1, os.cpu_count() or 1))
        with cf.ThreadPoolExecutor(jobs) as ex:
            list(ex.map(comp, todo))
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, LIB)
    return LIB


CHECKED_DIR = os.path.join(HERE, "_checked")


def build_checked(force: bool = False) -> str:
    """The bounds-checked variant (-DPOLARIS_CHECK) in paper_1412_1256_gb300/_checked/:
    kernels test their global-memory indices and record a bad one instead of touching it."""
    return build(force=force, out_dir=CHECKED_DIR, defines=("POLARIS_CHECK",))


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True))
