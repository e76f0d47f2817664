"""Build libsf.so (the CUDA library behind include/sf.h) in-tree for sm_103a.

nvcc compiles the translation units in parallel, then links one shared
library with the CUDA runtime linked statically.  Works the same on x86_64 and
aarch64 hosts (no host-architecture flags).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libsf.so")
SOURCES = ["sf_tableau.cu", "sf_tableau_warp.cu", "sf_frame.cu", "sf_api.cu", "sf_noalloc.cu", "sf_campaign.cu",
           "sf_gprog.cu", "sf_server.cu", "sf_multiframe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsf")


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "sf.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile and link; returns the path of libsf.so.  Rebuilds when a source
    is newer than the library."""
    with _lock:
        if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        os.makedirs(LIBDIR, exist_ok=True)
        cc = nvcc()
        common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread",
                         "-I", INCLUDE, "-I", CSRC]
        common += list(extra_flags)
        procs = []
        objs = []
        for src in SOURCES:
            obj = os.path.join(BUILD, src.replace(".cu", ".o"))
            objs.append(obj)
            cmd = [cc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        errors = []
        for cmd, p in procs:
            out, _ = p.communicate()
            if verbose or p.returncode:
                print(out.decode(errors="replace"))
            if p.returncode:
                errors.append(" ".join(cmd))
        if errors:
            raise RuntimeError("nvcc failed: " + "; ".join(errors))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static", "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
