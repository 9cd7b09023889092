"""Build liblogdet.so in-tree for sm_103a (nvcc for CUDA, g++ for host C++).

Translation units compile in parallel; the library links the CUDA runtime
statically so it loads without extra library paths.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "liblogdet.so")
BUILD = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["engine.cu", "engine_iter_f32.cu", "engine_iter_f64.cu", "static_scratch.cu", "matfree.cu"]
CXX_SOURCES = ["api.cpp", "bounds.cpp", "colouring.cpp", "fem.cpp", "hht.cpp"]
HEADERS = ["internal.h", "engine_device.cuh", "engine_iter.cuh", "engine_lean.cuh", "engine_csr.cuh",
           "engine_lean3d.cuh"]


def _cuda_home() -> str:
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _sources():
    return [os.path.join(CSRC, s) for s in CU_SOURCES + CXX_SOURCES + HEADERS] + [
        os.path.join(ROOT, "include", "logdet.h")]


def _stale() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    cuda = _cuda_home()
    nvcc = shutil.which("nvcc") or os.path.join(cuda, "bin", "nvcc")
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    jobs = []
    for s in CU_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     *inc, "-c", os.path.join(CSRC, s), "-o", o])
    for s in CXX_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", *inc,
                     "-I" + os.path.join(cuda, "include"), "-c", os.path.join(CSRC, s), "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for log in ex.map(run, jobs):
            if verbose and log:
                print(log)
    objs = [os.path.join(BUILD, s + ".o") for s in CU_SOURCES + CXX_SOURCES]
    tmp = OUT + ".%d.tmp" % os.getpid()
    run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
