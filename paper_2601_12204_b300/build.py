"""Builds libburgers.so in-tree with nvcc for sm_103a (B300).

Each .cu file under csrc/ is compiled to an object in csrc/_build/ (only when
its sources changed) and the objects are linked into
paper_2601_12204_b300/libburgers.so. `python -m paper_2601_12204_b300.build`
runs it; `--ptxas` prints the register / spill report of every kernel.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(CSRC, "_build")
LIB = os.path.join(HERE, "libburgers.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _digest(paths) -> str:
    h = hashlib.sha256()
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def _flags(ptxas: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                "--expt-relaxed-constexpr", "-Xcompiler", "-Wall"]
    if ptxas:
        f += ["-Xptxas", "-v"]
    return f


def build(force: bool = False, ptxas: bool = False, jobs: int = 0, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                     glob.glob(os.path.join(INCLUDE, "*.h")))
    hdr_digest = _digest(headers)
    objs = []
    todo = []
    for src in sources:
        tag = _digest([src]) + hdr_digest
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + f".{tag}.o")
        objs.append(obj)
        if force or ptxas or not os.path.exists(obj):
            todo.append((src, obj))

    def compile_one(job):
        src, obj = job
        cmd = [nvcc()] + _flags(ptxas) + ["-c", src, "-o", obj + ".tmp"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
        os.replace(obj + ".tmp", obj)
        return src, res.stdout + res.stderr

    if todo:
        n = jobs or min(len(todo), os.cpu_count() or 4)
        with cf.ThreadPoolExecutor(n) as ex:
            for src, out in ex.map(compile_one, todo):
                if verbose or ptxas:
                    sys.stdout.write(f"== {os.path.basename(src)}\n{out}")
    stale = not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs)
    if stale or force:
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, LIB)
    # drop objects of older source versions
    keep = set(objs)
    for o in glob.glob(os.path.join(BUILD, "*.o")):
        if o not in keep:
            os.remove(o)
    return LIB


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas", action="store_true", help="print -Xptxas -v output")
    ap.add_argument("-v", "--verbose", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, ptxas=a.ptxas, verbose=a.verbose))


if __name__ == "__main__":
    main()
