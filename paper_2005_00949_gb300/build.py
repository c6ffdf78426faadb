"""Build libgv.so in-tree with nvcc for sm_103a (GB300).

Translation units compile in parallel; the result is
paper_2005_00949_gb300/libgv.so (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libgv.so")
BUILD = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
SOURCES = ["gv_transport.cu", "gv_unit.cu", "gv_tables.cpp"]
HEADERS = ["gv_internal.h", "gv_device.cuh", "gv_state.cuh"]


def _needs(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, verbose: bool, min_blocks: int = 0, max_block: int = 0, maxnreg: int = 0,
             checks: bool = False) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    deps = [os.path.join(CSRC, src)] + [os.path.join(CSRC, h) for h in HEADERS] + \
        [os.path.join(ROOT, "include", "gv.h")]
    if not _needs(obj, deps):
        return obj
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        if min_blocks:
            cmd.insert(1, f"-DGV_MIN_BLOCKS={int(min_blocks)}")
        if max_block:
            cmd.insert(1, f"-DGV_MAX_BLOCK={int(max_block)}")
        if maxnreg:
            cmd.insert(1, f"-DGV_MAXNREG={int(maxnreg)}")
        if checks:
            cmd.insert(1, "-DGV_CHECKS")
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-c",
               os.path.join(CSRC, src), "-o", obj]
    subprocess.check_call(cmd)
    return obj


def build(force: bool = False, verbose: bool = False, min_blocks: int = 0, out: str = OUT,
          max_block: int = 0, maxnreg: int = 0, checks: bool = False) -> str:
    """Compile libgv.so.  min_blocks > 0 builds the step kernel with a register
    budget for that many resident blocks per SM of max_block threads (default
    256, the largest block_size it then accepts); maxnreg > 0 caps its
    registers per thread directly instead; checks=True compiles the index and
    state checks (GV_CHECKS) in.  Such variants go to their own build
    directory (pass `out` to keep the default library)."""
    global BUILD
    variant = min_blocks or max_block or maxnreg or checks
    build_dir = BUILD if not variant else BUILD + f"_mb{min_blocks}_{max_block}_{maxnreg}_{int(checks)}"
    os.makedirs(build_dir, exist_ok=True)
    if force:
        for f in os.listdir(build_dir):
            os.remove(os.path.join(build_dir, f))
    saved, BUILD = BUILD, build_dir
    try:
        with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
            objs = list(ex.map(lambda s: _compile(s, verbose, min_blocks, max_block, maxnreg, checks), SOURCES))
    finally:
        BUILD = saved
    if force or _needs(out, objs):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
