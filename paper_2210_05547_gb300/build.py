"""Build the CUDA libraries in-tree for sm_103a (GB300) with nvcc: ``_lib/libhyp.so`` for
five-species air and ``_lib/libhyp11.so`` for eleven-species air (ions and electrons), the same
sources compiled with the species count ``HYP_NSP`` 5 and 11.

Every translation unit of both variants is compiled in parallel, then each variant is linked as a
shared library that exports the C ABI declared in ``include/hyp.h``.
Usage: ``python -m paper_2210_05547_gb300.build``.
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
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libhyp.so")
LIB11 = os.path.join(OUT_DIR, "libhyp11.so")
VARIANTS = {5: LIB, 11: LIB11}
SOURCES = ["gas.cu", "lines.cu", "rhs.cu", "batch.cu", "serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include")]


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _compile(src, nsp, ptxas_verbose):
    obj = os.path.join(OUT_DIR, f"{os.path.splitext(src)[0]}_{nsp}.o")
    cmd = [nvcc(), *ARCH, *FLAGS, f"-DHYP_NSP={nsp}", "-c", os.path.join(CSRC, src), "-o", obj]
    if ptxas_verbose:
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src} ({nsp} species):\n{res.stderr}")
    return obj, res.stderr


def build(ptxas_verbose=False, quiet=True, variants=(5, 11)):
    os.makedirs(OUT_DIR, exist_ok=True)
    jobs = [(src, nsp) for nsp in variants for src in SOURCES]
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(lambda j: _compile(j[0], j[1], ptxas_verbose), jobs))
    if not quiet:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    for nsp in variants:
        objs = [r[0] for r, j in zip(results, jobs) if j[1] == nsp]
        lib = VARIANTS[nsp]
        tmp = lib + ".tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(ptxas_verbose="-v" in sys.argv, quiet=False))
