"""Build libt3f.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel to an object file under ``_build/`` and the
objects are linked into ``paper_1801_01928_gb300/libt3f.so`` (CUDA runtime linked
statically). Objects are rebuilt when a source or a header is newer than them.

    python -m paper_1801_01928_gb300.build [-v] [--ptxas-info]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libt3f.so")

SOURCES = ["api.cu", "sweep.cu", "gram.cu", "gather.cu", "matvec.cu", "orth.cu", "project.cu", "psweep.cu", "gram_tile.cu", "gram_tile_bwd.cu", "gram_groups.cu", "gram_mma.cu", "gram_mma_bwd.cu", "tangent.cu", "tgram_tc.cu", "probe.cu", "round.cu", "psweep_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found (CUDA toolkit required to build libt3f)")
    return path


def _headers() -> list[str]:
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs


def _compile(src: str, ptxas_info: bool) -> tuple[str, str]:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
    if ptxas_info:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(verbose: bool = False, ptxas_info: bool = False, force: bool = False) -> str:
    """Compile (if needed) and link libt3f.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    newest_hdr = max(os.path.getmtime(h) for h in _headers())
    todo = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        s_m = max(os.path.getmtime(os.path.join(CSRC, src)), newest_hdr)
        if force or ptxas_info or not os.path.exists(obj) or os.path.getmtime(obj) < s_m:
            todo.append(src)
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            for obj, log in ex.map(lambda s: _compile(s, ptxas_info), todo):
                if verbose or ptxas_info:
                    print(f"[t3f build] {os.path.basename(obj)}", file=sys.stderr)
                    if log:
                        print(log, file=sys.stderr)
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("-v", "--verbose", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true")
    ap.add_argument("--force", action="store_true")
    a = ap.parse_args()
    print(build(verbose=a.verbose, ptxas_info=a.ptxas_info, force=a.force))
