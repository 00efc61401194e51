"""Build libsparkling.so (sm_103a) in-tree with nvcc.

The translation units are compiled in parallel and linked into one shared
library with the CUDA runtime linked statically and cuFFT dynamically (the
node field of the fast attraction), exporting only the C ABI declared in
include/sparkling.h.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsparkling.so")
SOURCES = ["api.cu", "pairs.cu", "repulsion.cu", "repulsion_sym.cu", "project.cu", "noalloc.cu",
           "engine.cu", "field.cu", "driver.cu", "mesh.cu"]
HEADERS = ["kernels.h", "ptx.cuh", "pair_dev.cuh", "project_dev.cuh", "sym_dev.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsparkling.so")


def _flags(verbose_ptxas: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                "-I", os.path.join(ROOT, "include")]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile (when sources changed) and return the path of libsparkling.so."""
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "sparkling.h")]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + common):
            jobs.append((s, o))

    def compile_one(job):
        s, o = job
        cmd = [cc] + _flags(verbose_ptxas) + ["-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(s)}:\n{r.stderr}")
        return r.stderr

    logs = []
    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            logs = list(ex.map(compile_one, jobs))
    if verbose_ptxas:
        for line in "".join(logs).splitlines():
            print(line, file=sys.stderr)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(cc))), "lib64")
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcufft", "-Xlinker",
                                                              "-rpath," + cuda_lib]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
