"""Builds the in-tree CUDA library libsstep_cg.so for GB300 (sm_103a).

Each translation unit under csrc/ is compiled by nvcc in parallel into _build/, then linked
into paper_2512_09642_gb300/libsstep_cg.so. The Gram instantiation units (INSTANCED) are
compiled once per basis size s with -DSSTEP_INST_S=<s>: their cost grows steeply with s, so
one object per s, started largest first, keeps the longest compile near a minute. Objects are
reused when newer than their sources and the headers. Run
`python -m paper_2512_09642_gb300.build` or call build().
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsstep_cg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsstep_cg.so")


# translation units compiled once per basis size s, and the sizes
INSTANCED = {"k_gram_inst.cu": range(1, 33), "k_batch_gram_inst.cu": range(1, 17)}


def _units():
    """(source, object, extra flags, relative cost) for every compile job."""
    units = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        base = os.path.basename(src)[:-3]
        if os.path.basename(src) in INSTANCED:
            for s in INSTANCED[os.path.basename(src)]:
                units.append((src, os.path.join(BUILD, f"{base}_s{s:02d}.o"), [f"-DSSTEP_INST_S={s}"], s * s))
        else:
            units.append((src, os.path.join(BUILD, base + ".o"), [], 0))
    return units


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def _compile(nvcc, src, obj, extra, verbose):
    cmd = [nvcc] + ARCH + FLAGS + extra + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr[-4000:]}")
    return r.stderr


def build(verbose: bool = False, jobs: int = 0) -> str:
    """Compiles (if needed) and links the library; returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    hdr_time = max(os.path.getmtime(h) for h in _headers())
    todo, objs = [], []
    for s, o, extra, cost in _units():
        objs.append(o)
        if not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_time):
            todo.append((cost, s, o, extra))
    todo.sort(key=lambda u: -u[0])   # the longest compiles first
    jobs = jobs or min(len(todo) or 1, os.cpu_count() or 4)
    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = {ex.submit(_compile, nvcc, s, o, extra, verbose): os.path.basename(o) for _, s, o, extra in todo}
        for f in cf.as_completed(futs):
            logs.append((futs[f], f.result()))
    if verbose:
        for s, log in sorted(logs):
            sys.stderr.write(f"== {s}\n{log}")
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
