"""Compile the CUDA library (libriann.so) in-tree for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into ``paper_1508_07953_gb300/_lib/libriann.so``.  The translation units
whose kernels gather through table indices are compiled a second time with
-DRIANN_CHECKED (every gathered index tested before the access) and linked with
the others into ``_lib/libriann_checked.so``.  No GPU is needed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "libriann.so")
LIB_CHECKED = os.path.join(LIB_DIR, "libriann_checked.so")
CHECKED_SOURCES = ["sparse_query.cu", "dense_tc.cu", "anchor.cu"]
SOURCES = ["api.cu", "index_build.cu", "sparse_query.cu", "dense_tc.cu", "server.cu", "reconstruct.cu", "stack.cu", "cluster.cu", "unit.cu",
           "anchor.cu", "peaks.cu"]
HEADERS = sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "riann.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the RIANN CUDA library cannot be built")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    cc = nvcc()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src.replace(".cu", ".o"))
        if force or _stale(o, [s] + HEADERS):
            jobs.append([cc, *FLAGS, *extra_flags, "-c", s, "-o", o])
    for src in CHECKED_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src.replace(".cu", ".checked.o"))
        if force or _stale(o, [s] + HEADERS):
            jobs.append([cc, *FLAGS, *extra_flags, "-DRIANN_CHECKED", "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(OBJ, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-ldl"])
        os.replace(tmp, LIB)
    cobjs = [os.path.join(OBJ, s.replace(".cu", ".checked.o" if s in CHECKED_SOURCES else ".o")) for s in SOURCES]
    if force or jobs or _stale(LIB_CHECKED, cobjs):
        tmp = LIB_CHECKED + f".{os.getpid()}.tmp"
        run([cc, *ARCH, "-shared", "-o", tmp, *cobjs, "-ldl"])
        os.replace(tmp, LIB_CHECKED)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
