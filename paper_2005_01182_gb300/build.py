"""Build libotassign.so in-tree for sm_103a (nvcc, no cmake).

Every ``csrc/*.cu`` file is compiled to an object in parallel, then linked
with the shared CUDA runtime into ``paper_2005_01182_gb300/lib/libotassign.so``;
``client/served_client.cpp`` (a host-only client of the serving entry
points, used by the served benchmark) becomes ``lib/libotclient.so``.
Objects are rebuilt only when a source or header is newer.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libotassign.so")
CLIENT_SRC = os.path.join(PKG, "client", "served_client.cpp")
CLIENT_LIB = os.path.join(LIBDIR, "libotclient.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _headers_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.inc")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(f) for f in files), default=0.0)


def build(verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile and link; returns the path of the shared library."""
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr = _headers_mtime()
    flags = NVCC_FLAGS + (extra_flags or [])
    jobs = []
    for s in srcs:
        o = os.path.join(OBJ, os.path.basename(s)[:-3] + ".o")
        if not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            jobs.append([nvcc(), *ARCH, *flags, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    objs = [os.path.join(OBJ, os.path.basename(s)[:-3] + ".o") for s in srcs]
    if jobs or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([nvcc(), *ARCH, "-shared", "-cudart=shared", "-o", tmp, *objs, "-lpthread"])
        os.replace(tmp, LIB)
    # the serving client (host code only, calls the library's C-ABI)
    hdr_c = max(os.path.getmtime(CLIENT_SRC), os.path.getmtime(os.path.join(INCLUDE, "otassign.h")),
                os.path.getmtime(LIB))
    if not os.path.exists(CLIENT_LIB) or os.path.getmtime(CLIENT_LIB) < hdr_c:
        tmp = CLIENT_LIB + f".{os.getpid()}.tmp"
        run([os.environ.get("CXX", "g++"), "-O2", "-std=c++17", "-shared", "-fPIC", "-I", INCLUDE, CLIENT_SRC,
             "-o", tmp, "-L", LIBDIR, "-lotassign", "-Wl,-rpath,$ORIGIN", "-lpthread"])
        os.replace(tmp, CLIENT_LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
