"""Build libtwa.so (CUDA for sm_103a) in-tree with nvcc.

Translation units are compiled in parallel (one per FFT length plus the API,
misc and FP64 files) and linked into ``paper_2310_07119_gb300/libtwa.so``.
Objects go to ``paper_2310_07119_gb300/_build/``.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtwa.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers_digest() -> str:
    h = hashlib.sha1()
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cuh", ".h", ".inc")):
            h.update(open(os.path.join(CSRC, f), "rb").read())
    h.update(open(os.path.join(INCLUDE, "twa.h"), "rb").read())
    h.update(" ".join(ARCH + FLAGS + [platform.machine()]).encode())
    return h.hexdigest()


def source_digest() -> str:
    """Digest of the sources that define the line-pass kernels (the transform engine, the passes, their
    instantiations): identifies the kernels a profile was taken on.  Host-side API code is left out."""
    h = hashlib.sha1()
    for f in sorted(os.listdir(CSRC)):
        if f in ("fft_engine.cuh", "passes.cuh", "pipe.cuh", "passes_inst.inc") or \
                (f.startswith("passes_n") and f.endswith(".cu")):
            h.update(f.encode())
            h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()[:16]


def _compile(nvcc, src, dig):
    obj = os.path.join(BUILD, src[:-3] + ".o")
    stamp = obj + ".stamp"
    key = dig + hashlib.sha1(open(os.path.join(CSRC, src), "rb").read()).hexdigest()
    if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == key:
        return obj
    cmd = [nvcc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    with open(stamp, "w") as f:
        f.write(key)
    return obj


def build(verbose: bool = False, jobs: int = None) -> str:
    """Compile every CUDA source for sm_103a and link libtwa.so; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    dig = _headers_digest()
    srcs = _sources()
    jobs = jobs or max(1, min(len(srcs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, dig), srcs))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB} from {len(objs)} objects", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
