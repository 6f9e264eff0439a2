"""Build the CUDA library in-tree: nvcc for sm_103a only.

    python -m paper_2608_15390_b300.build [--force] [-v]

Compiles each csrc/*.cu whose object is missing or older than the source or
any header (every one with --force) in parallel, one nvcc per file, into
_lib/obj/, and links the objects into paper_2608_15390_b300/_lib/libpm_b300.so.  The ptxas
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


OBJ_DIR = os.path.join(LIB_DIR, "obj")


def headers():
    out = glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + glob.glob(os.path.join(HERE, "csrc", "*.h"))
    return out + glob.glob(os.path.join(ROOT, "include", "*.h"))


def _obj(src: str) -> str:
    return os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + ".o")


def _stale(src: str) -> bool:
    """An object is rebuilt when it is missing or older than its source or any header."""
    o = _obj(src)
    if not os.path.exists(o):
        return True
    t = os.path.getmtime(o)
    return any(os.path.getmtime(d) > t for d in [src, *headers()])


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in deps()) or any(_stale(s) for s in sources())


def _compile(src: str):
    tmp = _obj(src) + f".{os.getpid()}.tmp.o"
    r = subprocess.run([NVCC, *CFLAGS, "-c", "-o", tmp, src], capture_output=True, text=True)
    if r.returncode == 0:
        os.replace(tmp, _obj(src))
        with open(_obj(src)[:-2] + ".log", "w") as f:
            f.write(r.stdout + r.stderr)
    elif os.path.exists(tmp):
        os.unlink(tmp)
    return r


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the stale objects (every one with force), then link."""
    if not force and not needs_build():
        return LIB
    os.makedirs(OBJ_DIR, exist_ok=True)
    srcs = sources()
    todo = [s for s in srcs if force or _stale(s)]
    if todo:
        with ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 1))) as ex:
            results = list(ex.map(_compile, todo))
        for s, r in zip(todo, results):
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise RuntimeError("nvcc failed compiling " + s)
    objs = [_obj(s) for s in srcs]
    tmp = LIB + f".{os.getpid()}.tmp"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking " + LIB)
    os.replace(tmp, LIB)
    log = ""
    for s in srcs:
        lp = _obj(s)[:-2] + ".log"
        log += f"== {os.path.basename(s)}\n" + (open(lp).read() if os.path.exists(lp) else "")
    with open(os.path.join(LIB_DIR, "ptxas_info.txt"), "w") as f:
        f.write(log)
    if verbose:
        sys.stderr.write(log)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
