"""Build libdect.so (sm_103a) in-tree with nvcc; no cmake, one -gencode."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libdect.so")
# the same library with the index checks of DECT_CHECKED compiled in
LIB_CHECKED = os.path.join(OUT_DIR, "libdect_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libdect needs the CUDA 13 toolkit")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(lib: str = None) -> bool:
    libs = [lib] if lib else [LIB, LIB_CHECKED]
    for path in libs:
        if not os.path.exists(path):
            return False
        t = os.path.getmtime(path)
        if not all(os.path.getmtime(p) <= t for p in _deps()):
            return False
    return True


def _build_one(cc, lib, tag, flags, verbose, ex):
    objs = []

    def one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + tag + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    futs = [ex.submit(one, src) for src in _sources()]
    return lib, futs


def _link(cc, lib, objs):
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile every .cu in csrc/ in parallel and link libdect.so and
    libdect_checked.so (-DDECT_CHECKED).  Returns the path of libdect.so."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    variants = [(LIB, "", list(extra)), (LIB_CHECKED, ".chk", ["-DDECT_CHECKED", *extra])]
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        jobs = [_build_one(cc, lib, tag, flags, verbose, ex) for lib, tag, flags in variants]
        for lib, futs in jobs:
            _link(cc, lib, [f.result() for f in futs])
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
