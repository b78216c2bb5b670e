"""Compile libsddm.so (sm_103a) in-tree with nvcc: csrc/*.cu and csrc/*.cpp -> _build/."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsddm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs + [os.path.join(ROOT, "include", "sddm.h")]


def _flags(extra=()):
    return ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]


def _compile(src, extra):
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    cmd = [NVCC, *_flags(extra), "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Build libsddm.so if any source is newer than it; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    srcs = _sources()
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(f) <= t for f in srcs + _headers() + [__file__]):
            return LIB
    jobs = max(1, min(len(srcs), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), srcs))
    if verbose:
        for _, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC, "-shared", *ARCH, "-o", tmp, *[o for o, _ in results], "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    # --force: rebuild; --ptxas: print register/spill use; -DNAME=VALUE: compile-time
    # kernel options (e.g. -DSDDM_TRACE_MIN_BLOCKS=10 -DSDDM_TRACE_SPEC=1)
    extra = (["-Xptxas", "-v"] if "--ptxas" in sys.argv else []) + [a for a in sys.argv[1:] if a.startswith("-D")]
    print(build(force="--force" in sys.argv or any(a.startswith("-D") for a in sys.argv[1:]), verbose=True,
                extra=extra))
