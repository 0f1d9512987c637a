"""Build libhelm.so in-tree for sm_103a (nvcc, one translation unit per source,
compiled in parallel, then linked).  Used by __graft_entry__.build()."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhelm.so")
SOURCES = ["stencil.cu", "blas.cu", "bicg32.cu", "tb.cu", "adjoint.cu", "nn.cu", "batch.cu", "helm_api.cu", "noalloc.cu",
           "mg.cu", "gemm_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, extra, build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    tu = ["-DHELM_TU_ID=%d" % SOURCES.index(src)] if src in SOURCES else []
    cmd = [nvcc(), *ARCH, *FLAGS, *tu, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


LIB_CHECKED = os.path.join(HERE, "libhelm_checked.so")


def build(verbose: bool = False, extra=(), checked: bool = False) -> str:
    """libhelm.so; with checked=True also libhelm_checked.so, the bounds-checked
    variant (-DHELM_CHECKED), compiled in the same parallel pass."""
    variants = [(BUILD, LIB, list(extra))]
    if checked:
        variants.append((BUILD + "_checked", LIB_CHECKED, list(extra) + ["-DHELM_CHECKED"]))
    jobs = []
    for bdir, _, ex_flags in variants:
        os.makedirs(bdir, exist_ok=True)
        jobs += [(src, ex_flags, bdir) for src in SOURCES]
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(lambda j: _compile(*j), jobs))
    for vi, (bdir, lib, _) in enumerate(variants):
        vobjs = objs[vi * len(SOURCES):(vi + 1) * len(SOURCES)]
        cmd = [nvcc(), *ARCH, "-shared", "-o", lib + ".tmp", *vobjs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(lib + ".tmp", lib)
        if verbose:
            print("built", lib)
    return LIB


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if a != "--checked"]
    build(verbose=True, extra=args, checked="--checked" in sys.argv[1:])
