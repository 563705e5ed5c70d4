"""Build libvmt.so (CUDA kernels for sm_103a + the C ABI) in-tree.

    python -m paper_2309_16682_gb300.build [--force]

Each translation unit is compiled by its own nvcc/g++ process in parallel, then
linked into paper_2309_16682_gb300/_build/libvmt.so.  Only one -gencode target
is built: sm_103a (GB300).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libvmt.so")

CUDA_SOURCES = ["gen_mt.cu", "gen_mt32.cu", "gen_mt64.cu", "gen_mtc32.cu", "gen_mtc64.cu", "gen_sfmt.cu", "gen_sfmt_m1.cu", "gen_sfmt_m2.cu", "gen_sfmt_m4.cu", "gen_sfmt_m8.cu",
                "gen_sfmt_m16.cu", "jump.cu", "vmt_capi.cu", "noalloc.cu", "serve.cu", "diag.cu", "scalar.cu", "tgfsr.cu"]
CXX_SOURCES = ["gf2poly.cpp"]
HEADERS = ["vmt_device.cuh", "gen_mt.cuh", "gen_mt_kernel.cuh", "gen_mtc.cuh", "vmt_internal.hpp", "gen_args.hpp", "gf2poly.hpp", "bulk.cuh", "gen_sfmt.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvmt.so")
    return p


def _inputs():
    files = [os.path.join(CSRC, f) for f in CUDA_SOURCES + CXX_SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "vmt.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stderr


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nv = nvcc()
    common = ["-O3", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    jobs = []
    objs = []
    for f in CUDA_SOURCES:
        o = os.path.join(OUT, f + ".o")
        objs.append(o)
        cmd = [nv, *ARCH, "-lineinfo", *common, "-Xcompiler", "-fPIC", "-c", os.path.join(CSRC, f), "-o", o]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        jobs.append(cmd)
    cxx = shutil.which("g++") or "c++"
    for f in CXX_SOURCES:
        o = os.path.join(OUT, f + ".o")
        objs.append(o)
        jobs.append([cxx, "-O3", "-std=c++17", "-fPIC", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                     "-c", os.path.join(CSRC, f), "-o", o])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_compile, jobs))
    if verbose or ptxas_info:
        for l in logs:
            if l:
                sys.stderr.write(l)
    tmp = LIB + f".tmp{os.getpid()}"
    _compile([nv, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true")
    args = ap.parse_args()
    print(build(force=args.force, verbose=True, ptxas_info=args.ptxas_info))
