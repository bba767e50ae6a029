"""Compile the CUDA library ``libmoc3d.so`` in-tree for sm_103a.

Host C++ (moc_host.cpp) is compiled by g++ without fused multiply-add
contraction; the CUDA translation units by nvcc with a single
``-gencode arch=compute_103a,code=sm_103a``.  Units compile in parallel.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmoc3d.so")
INCLUDE = os.path.join(ROOT, "include")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["moc_kernels.cu", "moc_sweep.cu", "moc_sweep_f32g1.cu", "moc_sweep_f32g2.cu", "moc_sweep_f32g2m.cu",
              "moc_sweep_f32g4.cu", "moc_sweep_f64.cu", "moc_api.cu", "moc_static.cu", "moc_peak.cu",
              "moc_server.cu", "moc_tune.cu", "moc_trace.cu",
              "moc_sweep_ol.cu"]
# per-file nvcc flags: the device 2D tracer must round like the host tracer
CU_FLAGS = {"moc_trace.cu": ["-fmad=false"]}
CPP_SOURCES = ["moc_host.cpp"]


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "moc.h")]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(force: bool = False, verbose: bool = False, extra_nvcc=()) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    objs = []
    for f in CU_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append([NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC,
                     *CU_FLAGS.get(f, []), *extra_nvcc, "-c", os.path.join(CSRC, f), "-o", o])
    for f in CPP_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
                     "-I", INCLUDE, "-I", CSRC, "-I", "/usr/local/cuda/include",
                     "-c", os.path.join(CSRC, f), "-o", o])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    tmp = LIB + ".tmp"
    _run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra_nvcc=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)
