"""Builds the CUDA library paper_2408_04875_gb300/libubqp.so for sm_103a.

Each translation unit under csrc/ is compiled by its own nvcc process (in parallel),
then linked into one shared library with a plain C ABI (include/ubqp.h).  No torch
headers are involved; the library only needs the CUDA runtime and driver.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libubqp.so")
BUILD = os.path.join(ROOT, "_build")
SOURCES = ["engine.cu", "tick_gemv.cu", "lane_loop.cu", "solo.cu", "tick_update.cu", "init.cu", "noalloc.cu",
           "tc_gemm.cu"]
# the lane loop and the single-lane kernel read, within one launch, lane vectors that CTAs on
# other SMs wrote: their plain loads are cached in L2 only
EXTRA = {"lane_loop.cu": ["-Xptxas", "-dlcm=cg"], "solo.cu": ["-Xptxas", "-dlcm=cg"]}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libubqp.so")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
                   "--expt-relaxed-constexpr"] + list(extra)


def _stale(objs) -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "ubqp.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in srcs]
    if not force and not _stale(objs):
        return OUT
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src, obj):
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(list(extra) + EXTRA.get(src, []))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        logs = list(ex.map(compile_one, srcs, objs))
    if verbose or ptxas_info:
        for s, lg in zip(srcs, logs):
            if lg.strip():
                print(f"--- {s}\n{lg}", file=sys.stderr)
    tmp = OUT + f".{os.getpid()}.tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
