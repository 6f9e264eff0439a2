"""Build the CUDA library in-tree: nvcc for sm_103a only.

    python -m paper_2608_15390_b300.build [--force] [-v]

Compiles every csrc/*.cu to an object in parallel (one nvcc per file) and
links them into paper_2608_15390_b300/_lib/libpm_b300.so.  The ptxas
resource report (registers, spills, shared memory per kernel) is kept in
_lib/ptxas_info.txt.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "libpm_b300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = [*ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-Xptxas", "-v"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def deps():
    pats = ["*.cu", "*.cuh", "*.h"]
    out = []
    for p in pats:
        out += glob.glob(os.path.join(HERE, "csrc", p))
    out += glob.glob(os.path.join(ROOT, "include", "*.h"))
    return out


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in deps())


def _compile(src: str, obj: str):
    return subprocess.run([NVCC, *CFLAGS, "-c", "-o", obj, src], capture_output=True, text=True)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(LIB_DIR, exist_ok=True)
    srcs = sources()
    tag = f"{os.getpid()}"
    objs = [os.path.join(LIB_DIR, os.path.basename(s)[:-3] + f".{tag}.o") for s in srcs]
    try:
        with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
            results = list(ex.map(_compile, srcs, objs))
        log = ""
        for s, r in zip(srcs, results):
            log += f"== {os.path.basename(s)}\n{r.stdout}{r.stderr}"
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise RuntimeError("nvcc failed compiling " + s)
        tmp = LIB + f".{tag}.tmp"
        r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("nvcc failed linking " + LIB)
        if verbose:
            sys.stderr.write(log)
        os.replace(tmp, LIB)
        with open(os.path.join(LIB_DIR, "ptxas_info.txt"), "w") as f:
            f.write(log)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.unlink(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
