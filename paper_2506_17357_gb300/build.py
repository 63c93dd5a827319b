"""Build libtga.so (CUDA kernels + C-ABI) in-tree for sm_103a with nvcc.

Translation units are compiled in parallel and linked into
``paper_2506_17357_gb300/libtga.so``.  The same sources compiled with
``-DTGA_BOUNDS_CHECK`` give ``libtga_check.so``, the index-checked build
(every indexed device access checked against its array's extent; the
binding loads it when TGA_INDEX_CHECKS=1).  Objects go to ``_build/`` and
``_build_check/`` next to this file (git-ignored).  A library is rebuilt
only when a source or header is newer than it.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtga.so")
BUILD_DIR_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libtga_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The batched kernel reads job state that other SMs rewrite during the same
# launch: its global loads must bypass the (non-coherent) L1.
PER_FILE_FLAGS = {"tga_batch.cu": ["-Xptxas", "-dlcm=cg"], "tga_persist.cu": ["-Xptxas", "-dlcm=cg"]}


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtga")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(lib) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _sources() + _headers() + [__file__])


def build(force: bool = False, verbose: bool = False, extra_flags=None, check: bool = True) -> str:
    """Build libtga.so and (check=True) libtga_check.so; returns libtga.so's path."""
    variants = [(LIB, BUILD_DIR, [])]
    if check:
        variants.append((LIB_CHECK, BUILD_DIR_CHECK, ["-DTGA_BOUNDS_CHECK"]))
    variants = [v for v in variants if force or _stale(v[0])]
    if not variants:
        return LIB
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", INCLUDE, "-I", CSRC] + list(extra_flags or [])

    def compile_one(job):
        src, bdir, flags = job
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + common + flags + PER_FILE_FLAGS.get(os.path.basename(src), []) + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    jobs = []
    for _, bdir, flags in variants:
        os.makedirs(bdir, exist_ok=True)
        jobs += [(src, bdir, flags) for src in _sources()]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, jobs))
    for lib, bdir, _ in variants:
        mine = [o for o, (_, b, _) in zip(objs, jobs) if b == bdir]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + mine + ["-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
