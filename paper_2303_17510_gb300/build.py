"""Build libhd.so (CUDA kernels + C ABI) in-tree for sm_103a.

Every .cu file under csrc/ is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and linked
into ``_build/libhd.so``.  Object files are reused when neither the sources
(including headers) nor the flags changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libhd.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "--expt-relaxed-constexpr",
         "-I" + CSRC, "-I" + INCLUDE]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhd")


_INC = re.compile(r'^\s*#\s*include\s+"([^"]+)"', re.M)


def _deps_digest(src: str) -> str:
    """Digest of a source and every quoted header it includes, transitively."""
    h = hashlib.sha256()
    seen, todo = set(), [os.path.abspath(src)]
    while todo:
        p = todo.pop()
        if p in seen or not os.path.exists(p):
            continue
        seen.add(p)
        txt = open(p, "rb").read()
        h.update(p.encode())
        h.update(txt)
        for inc in _INC.findall(txt.decode("utf-8", "replace")):
            todo.append(os.path.abspath(os.path.join(os.path.dirname(p), inc)))
    return h.hexdigest()


def _compile(src: str, hdr: str, extra) -> str:
    base = os.path.splitext(os.path.basename(src))[0]
    key = hashlib.sha256((_deps_digest(src) + " ".join(ARCH + FLAGS + extra)).encode()).hexdigest()[:16]
    obj = os.path.join(OUT_DIR, f"{base}.{key}.o")
    if not os.path.exists(obj):
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, obj)
    return obj


def build(verbose: bool = False, jobs: int | None = None, extra=None) -> str:
    """Builds (or reuses) libhd.so; concurrent callers (one per rank) are
    serialized by a file lock, so only the first compiles."""
    os.makedirs(OUT_DIR, exist_ok=True)
    import fcntl
    with open(os.path.join(OUT_DIR, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        try:
            return _build_locked(verbose, jobs, extra)
        finally:
            fcntl.flock(lk, fcntl.LOCK_UN)


def _build_locked(verbose, jobs, extra) -> str:
    extra = list(extra or [])
    # the kernel instantiation units take longest: start them first
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")), key=lambda p: ("hd_conv1d_" not in p, p))
    hdr = ""
    jobs = jobs or max(1, min(len(srcs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, hdr, extra), srcs))
    key = hashlib.sha256(("".join(objs)).encode()).hexdigest()[:16]
    stamp = os.path.join(OUT_DIR, "libhd.stamp")
    if os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == key:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(key)
    # drop stale objects of earlier source versions
    keep = set(objs)
    for o in glob.glob(os.path.join(OUT_DIR, "*.o")):
        if o not in keep:
            try:
                os.remove(o)
            except OSError:
                pass
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
