"""Build libmdk.so (the CUDA path) in-tree with nvcc for sm_103a.

Each .cu file under csrc/ is compiled to an object in parallel, then linked
into paper_2511_22951_gb300/libmdk.so.  Nothing is installed anywhere else.

Freshness: a stamp file beside the library holds the sha256 of every source
and header, the compiler flags and `nvcc --version`; the library is rebuilt
whenever the stamp is missing or differs (file times are not trusted: a copy
or a checkout can make a stale library look newer than its sources).
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmdk.so")
STAMP = LIB + ".stamp"
# debug build: the kernels' index checks compiled in (MDK_DEBUG), its own
# objects, library and stamp
DEBUG_LIB = os.path.join(HERE, "libmdk_debug.so")
DEBUG_FLAGS = ("-DMDK_DEBUG=1",)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    return sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")] + \
        [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]


def fingerprint(extra=()) -> str:
    """sha256 over the sources and headers (names and contents), the flags
    and the compiler's version string."""
    h = hashlib.sha256()
    for d in sorted(_deps()):
        h.update(os.path.relpath(d, ROOT).encode())
        with open(d, "rb") as f:
            h.update(f.read())
    h.update(" ".join([*ARCH, *NVCC_FLAGS, *extra]).encode())
    try:
        v = subprocess.run([nvcc(), "--version"], capture_output=True, text=True).stdout
    except OSError:
        v = "no nvcc"
    h.update(v.encode())
    return h.hexdigest()


def up_to_date(extra=(), lib=LIB) -> bool:
    stamp = lib + ".stamp"
    if not (os.path.exists(lib) and os.path.exists(stamp)):
        return False
    with open(stamp) as f:
        return f.read().strip() == fingerprint(extra)


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    """Build libmdk.so (debug=True: libmdk_debug.so with the index checks)."""
    lib = DEBUG_LIB if debug else LIB
    extra = tuple(extra) + (DEBUG_FLAGS if debug else ())
    if not force and up_to_date(extra, lib):
        return lib
    stamp = fingerprint(extra)
    bdir = BUILD + ("_debug" if debug else "")
    os.makedirs(bdir, exist_ok=True)
    objs = []

    def one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(one, sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl",
           "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(lib + f".stamp.tmp{os.getpid()}", "w") as f:
        f.write(stamp + "\n")
    os.replace(lib + f".stamp.tmp{os.getpid()}", lib + ".stamp")
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else (),
                debug="--debug" in sys.argv))
