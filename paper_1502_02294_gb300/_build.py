"""Build liblc.so (the CUDA path) in-tree for sm_103a.

Every translation unit is compiled by nvcc with
``-gencode arch=compute_103a,code=sm_103a`` in parallel, then linked into
``paper_1502_02294_gb300/liblc.so``.  The FFT pass kernels are instantiated
once per supported grid size (one object per N).  No CPU fallback exists:
without this library the package refuses to work.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblc.so")
SIZES = (8, 16, 32, 64, 96, 128, 192, 256, 384, 512)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-Xcompiler", "-fno-fast-math", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblc")
    return cand


def _jobs():
    nv = _nvcc()
    jobs = []
    for src in ("lc_api.cu", "lc_device.cu", "lc_noalloc.cu"):
        path = os.path.join(CSRC, src)
        if os.path.exists(path):
            jobs.append(([nv, *ARCH, *NVCC_FLAGS, "-c", path, "-o", os.path.join(BUILD, src + ".o")], path))
    host = os.path.join(CSRC, "lc_host.cpp")
    jobs.append(([nv, *NVCC_FLAGS, "-x", "c++", "-c", host, "-o", os.path.join(BUILD, "lc_host.o")], host))
    inst = os.path.join(CSRC, "lc_fft_inst.cu")
    for n in SIZES:
        jobs.append(([nv, *ARCH, *NVCC_FLAGS, f"-DLC_N={n}", "-c", inst, "-o",
                      os.path.join(BUILD, f"lc_fft_{n}.o")], inst))
    return jobs


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    for d in (CSRC, os.path.join(HERE, "..", "include")):
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs = _jobs()

    def run(cmd):
        r = subprocess.run(cmd[0], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd[0])}\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return cmd[0][-1]

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(run, jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
