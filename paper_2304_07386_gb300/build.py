"""In-tree build of the SMM C-ABI library (libsmm.so) for sm_103a.

Translation units are compiled in parallel with nvcc and linked into
``paper_2304_07386_gb300/_lib/libsmm.so``.  A unit is rebuilt when its
source, a header it includes, or this file is newer than its object.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libsmm.so")
UNITS = ["setup.cpp", "amg.cpp", "sweep.cu", "moments.cu", "mg.cu", "cgsmm.cu", "api.cu", "cnn.cu", "noalloc.cu"]
HEADERS = [os.path.join(CSRC, h) for h in ("kernels.cuh", "setup.hpp", "amg.hpp", "blockops.cuh", "dfloat.cuh")] + [os.path.join(ROOT, "include", "smm.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(src: str, obj: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src, __file__] + HEADERS
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for u in UNITS:
        src = os.path.join(CSRC, u)
        obj = os.path.join(OUT, u + ".o")
        if _stale(src, obj):
            lang = ["-x", "cu"] if u.endswith(".cu") else ["-x", "c++"]
            jobs.append((u, [nvcc] + FLAGS + ARCH + lang + ["-c", src, "-o", obj]))

    def run(job):
        name, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(f"[smm build] {' '.join(cmd)}\n{r.stdout}{r.stderr}")
        return name, r.returncode

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        results = list(ex.map(run, jobs))
    bad = [n for n, rc in results if rc]
    if bad:
        raise RuntimeError(f"nvcc failed for {bad}")
    objs = [os.path.join(OUT, u + ".o") for u in UNITS]
    if jobs or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB] + objs + ["-Xcompiler", "-fopenmp", "-lgomp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError(f"link failed:\n{r.stdout}{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
