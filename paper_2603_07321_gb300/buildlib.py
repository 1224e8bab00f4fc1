"""Build the CUDA library libpta.so for sm_103a with nvcc (in-tree).

Each translation unit is compiled in parallel; the objects are linked into
paper_2603_07321_gb300/_lib/libpta.so.  No CMake, no torch extension
machinery: the library is plain CUDA C++ behind the C ABI of include/pta.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_lib")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libpta.so")
# debug build: every index and count tested before use (-DPTA_CHECK=1)
OBJ_CHECK = os.path.join(PKG, "_build_check")
LIB_CHECK = os.path.join(OUT, "libpta_check.so")
SOURCES = ["pta_api.cu", "k_setup.cu", "k_neigh.cu", "k_pair_f32.cu", "k_pair_f64.cu",
           "k_noalloc.cu", "k_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I" + INC,
         "-I" + CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compile (what is stale of) the library; returns its path.  check=True
    builds the debug variant libpta_check.so (PTA_CHECK=1) instead."""
    obj_dir, lib = (OBJ_CHECK, LIB_CHECK) if check else (OBJ, LIB)
    flags = FLAGS + (["-DPTA_CHECK=1"] if check else [])
    os.makedirs(OUT, exist_ok=True)
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(INC, "pta.h"))
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(obj_dir, src + ".o")
        if force or _stale(o, [s] + headers):
            jobs.append((s, o))

    def compile_one(job):
        s, o = job
        cmd = [nvcc] + ARCH + flags + ["-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s" % (s, r.stderr))
        if verbose:
            sys.stderr.write(r.stderr)
        return o

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(compile_one, jobs))
    objs = [os.path.join(obj_dir, src + ".o") for src in SOURCES]
    if force or jobs or _stale(lib, objs):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s" % r.stderr)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, check="--check" in sys.argv))
