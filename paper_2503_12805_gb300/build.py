"""Build the C-ABI shared library ``libwke.so`` in-tree for sm_103a.

Each translation unit is compiled in parallel (nvcc for the CUDA sources,
g++ for the host plan code) and linked with nvcc into
``paper_2503_12805_gb300/libwke.so``.  Objects go to ``_build/``.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libwke.so")
# the bounds-checked debug build (-DWKE_CHECK)
BUILD_CHECK = os.path.join(PKG, "_build_check")
LIB_CHECK = os.path.join(PKG, "libwke_check.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + INCLUDE, "-I" + CSRC]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-I" + INCLUDE, "-I" + CSRC]

CUDA_SOURCES = ["wke_api.cu", "wke_kernels_f32.cu", "wke_kernels_f64.cu", "wke_fused64_f32.cu", "wke_fused_f32.cu", "wke_noalloc.cu", "wke_peak.cu", "wke_server.cu"]
CXX_SOURCES = ["wke_plan.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd):
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + proc.stdout + proc.stderr)
    return proc.stdout + proc.stderr


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def _jobs(build_dir, defines, force, extra_nvcc, nvcc, headers):
    os.makedirs(build_dir, exist_ok=True)
    jobs, objs = [], []
    for src in CUDA_SOURCES:
        sp = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src + ".o")
        objs.append(o)
        if force or _stale(o, [sp] + headers):
            jobs.append([nvcc] + ARCH + NVCC_FLAGS + list(defines) + list(extra_nvcc) + ["-c", sp, "-o", o])
    for src in CXX_SOURCES:
        sp = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src + ".o")
        objs.append(o)
        if force or _stale(o, [sp] + headers):
            jobs.append(["g++"] + CXX_FLAGS + list(defines) + ["-c", sp, "-o", o])
    return jobs, objs


def build(verbose: bool = False, force: bool = False, extra_nvcc=(), check: bool = True) -> str:
    """Compile and link libwke.so (and, with `check`, the bounds-checked
    libwke_check.so); all translation units compile in parallel.  Returns
    the path of libwke.so."""
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "wke.h"))
    variants = [(BUILD, LIB, ())] + ([(BUILD_CHECK, LIB_CHECK, ("-DWKE_CHECK",))] if check else [])
    plans = [(lib_path,) + _jobs(d, defs, force, extra_nvcc, nvcc, headers) for d, lib_path, defs in variants]
    jobs = [j for _, js, _ in plans for j in js]
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for out in ex.map(_run, jobs):
            if verbose and out.strip():
                print(out)
    for lib_path, js, objs in plans:
        if force or js or _stale(lib_path, objs):
            _run([nvcc] + ARCH + ["-shared", "-o", lib_path] + objs)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
