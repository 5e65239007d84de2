"""Build step: generate the per-process device code, compile every CUDA translation
unit for sm_103a with nvcc (in parallel), and link libme_b300.so in-tree.

    python -m paper_2312_02898_b300.build [--force] [--jobs N]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import re
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
GEN = os.path.join(CSRC, "generated")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libme_b300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                 "-I", INCLUDE, "-I", CSRC]


_INCLUDE_RE = re.compile(r'^\s*#\s*include\s+"([^"]+)"', re.M)


def _deps(cu):
    """the source and every local header it includes, followed recursively"""
    seen, todo = set(), [os.path.abspath(cu)]
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(f):
            continue
        seen.add(f)
        for inc in _INCLUDE_RE.findall(open(f).read()):
            for base in (os.path.dirname(f), CSRC, INCLUDE):
                cand = os.path.normpath(os.path.join(base, inc))
                if os.path.exists(cand):
                    todo.append(cand)
                    break
    return sorted(seen)


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(cu, obj, log):
    t = time.time()
    r = subprocess.run([NVCC] + CFLAGS + ["-c", cu, "-o", obj + ".tmp"], capture_output=True, text=True)
    with open(log, "w") as f:
        f.write(r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {cu}:\n{r.stderr[-4000:]}")
    os.replace(obj + ".tmp", obj)
    return cu, time.time() - t


def build(force: bool = False, jobs: int | None = None, verbose: bool = True) -> str:
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2312_02898_b300.gen.emit import generate_all
    os.makedirs(BUILD, exist_ok=True)
    generate_all(GEN)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    skip = [t for t in os.environ.get("ME_B300_SKIP", "").split(",") if t]
    sources = [s for s in sources if os.path.basename(s)[:-3] not in (f"proc_{t}" for t in skip)]

    def size(cu):
        g = os.path.join(GEN, os.path.basename(cu)[:-3] + ".cuh")
        return os.path.getsize(g) if os.path.exists(g) else 0

    sources.sort(key=lambda s: -size(s))  # longest compile first
    objs, todo = [], []
    for cu in sources:
        name = os.path.basename(cu)[:-3]
        obj = os.path.join(BUILD, name + ".o")
        objs.append(obj)
        if force or _stale(obj, _deps(cu)):
            todo.append((cu, obj, os.path.join(BUILD, name + ".ptxas.log")))
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for cu, dt in ex.map(lambda x: _compile(*x), todo):
                if verbose:
                    print(f"[build] {os.path.basename(cu)} {dt:.1f}s", flush=True)
    if force or todo or _stale(LIB, objs):
        tmp = LIB + ".tmp"
        subprocess.check_call([NVCC] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, LIB)
        if verbose:
            print(f"[build] linked {LIB}", flush=True)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    args = ap.parse_args()
    build(force=args.force, jobs=args.jobs)
