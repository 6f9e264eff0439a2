"""Build the CUDA library in-tree: nvcc for sm_103a only.

    python -m paper_2608_15390_b300.build [--force] [-v] [--debug | --all]

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
LIB_DEBUG = os.path.join(LIB_DIR, "libpm_b300_debug.so")
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


def _variant(debug: bool):
    """(library, object directory, extra flags) of the release or PM_DEBUG build."""
    if debug:
        return LIB_DEBUG, os.path.join(LIB_DIR, "obj_debug"), ["-DPM_DEBUG"]
    return LIB, os.path.join(LIB_DIR, "obj"), []


def headers():
    out = glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + glob.glob(os.path.join(HERE, "csrc", "*.h"))
    return out + glob.glob(os.path.join(ROOT, "include", "*.h"))


def _obj(src: str, debug: bool = False) -> str:
    return os.path.join(_variant(debug)[1], os.path.basename(src)[:-3] + ".o")


def _stale(src: str, debug: bool = False) -> bool:
    """An object is rebuilt when it is missing or older than its source or any header."""
    o = _obj(src, debug)
    if not os.path.exists(o):
        return True
    t = os.path.getmtime(o)
    return any(os.path.getmtime(d) > t for d in [src, *headers()])


def needs_build(debug: bool = False) -> bool:
    lib = _variant(debug)[0]
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps()) or any(_stale(s, debug) for s in sources())


def _compile(src: str, debug: bool = False):
    obj = _obj(src, debug)
    tmp = obj + f".{os.getpid()}.tmp.o"
    r = subprocess.run([NVCC, *CFLAGS, *_variant(debug)[2], "-c", "-o", tmp, src], capture_output=True, text=True)
    if r.returncode == 0:
        os.replace(tmp, obj)
        with open(obj[:-2] + ".log", "w") as f:
            f.write(r.stdout + r.stderr)
    elif os.path.exists(tmp):
        os.unlink(tmp)
    return r


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile the stale objects (every one with force), then link.  debug:
    the PM_DEBUG variant (bounds-checked matrix views in the trajectory
    kernels) into _lib/libpm_b300_debug.so."""
    lib, obj_dir, _ = _variant(debug)
    if not force and not needs_build(debug):
        return lib
    os.makedirs(obj_dir, exist_ok=True)
    srcs = sources()
    todo = [s for s in srcs if force or _stale(s, debug)]
    if todo:
        with ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 1))) as ex:
            results = list(ex.map(lambda s: _compile(s, debug), todo))
        for s, r in zip(todo, results):
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise RuntimeError("nvcc failed compiling " + s)
    objs = [_obj(s, debug) for s in srcs]
    tmp = lib + f".{os.getpid()}.tmp"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking " + lib)
    os.replace(tmp, lib)
    log = ""
    for s in srcs:
        lp = _obj(s, debug)[:-2] + ".log"
        log += f"== {os.path.basename(s)}\n" + (open(lp).read() if os.path.exists(lp) else "")
    with open(os.path.join(LIB_DIR, "ptxas_info_debug.txt" if debug else "ptxas_info.txt"), "w") as f:
        f.write(log)
    if verbose:
        sys.stderr.write(log)
    return lib


def build_all(force: bool = False) -> None:
    """The release and the PM_DEBUG libraries, side by side."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        for f in [ex.submit(build, force, False, d) for d in (False, True)]:
            f.result()


if __name__ == "__main__":
    if "--all" in sys.argv:
        build_all(force="--force" in sys.argv)
        print(LIB, LIB_DEBUG)
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
