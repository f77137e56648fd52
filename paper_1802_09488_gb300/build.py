"""Builds the native library libagj.so in-tree (paper_1802_09488_gb300/_build).

CUDA sources are compiled by nvcc for sm_103a only
(-gencode arch=compute_103a,code=sm_103a) with -fmad=false, so FP64 cell ids
and the PIP orientation round exactly as the host spec does; host C++ is
compiled by g++ with -ffp-contract=off for the same reason.  Translation
units compile in parallel; the whole build takes well under a minute.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libagj.so")
ROOT = os.path.dirname(HERE)

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CXXFLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-pthread", "-Wall",
            f"-I{CUDA_HOME}/include", f"-I{ROOT}/include"]
NVCCFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", *ARCH, "-Xcompiler", "-fPIC,-ffp-contract=off",
             f"-I{ROOT}/include", "--expt-relaxed-constexpr"]

CU_SOURCES = ["agj_kernels.cu", "agj_batch.cu"]
CXX_SOURCES = ["agj_build.cpp", "agj_model.cpp", "agj_capi.cpp", "agj_server.cpp"]


def _sources():
    return [os.path.join(CSRC, f) for f in CU_SOURCES + CXX_SOURCES]


def _headers():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))] + \
        [os.path.join(ROOT, "include", "agj.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _sources() + _headers() + [os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False) -> str:
    """Builds libagj.so; extra nvcc flags may come from $AGJ_NVCC_EXTRA (for
    example -DAGJ_PROBE_MIN_BLOCKS=6)."""
    if not force and up_to_date():
        return LIB
    if not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}; the CUDA toolkit is required to build libagj.so")
    os.makedirs(OUT, exist_ok=True)
    procs, objs = [], []
    for f in CU_SOURCES:
        obj = os.path.join(OUT, f.replace(".cu", ".o"))
        cmd = [NVCC, *NVCCFLAGS, *os.environ.get("AGJ_NVCC_EXTRA", "").split(), "-c", os.path.join(CSRC, f), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    cxx = shutil.which("g++") or "g++"
    for f in CXX_SOURCES:
        obj = os.path.join(OUT, f.replace(".cpp", ".o"))
        cmd = [cxx, *CXXFLAGS, "-c", os.path.join(CSRC, f), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((cmd, text))
        elif verbose and text.strip():
            print(text, file=sys.stderr)
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + t for c, t in failed)
        raise RuntimeError("libagj build failed:\n" + msg)
    tmp = LIB + f".tmp{os.getpid()}"
    link = [NVCC, "-shared", *ARCH, "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libagj link failed:\n" + " ".join(link) + "\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
