"""Builds libpmmm.so (the CUDA kernels and the C ABI of include/pmmm.h) in-tree
for sm_103a with nvcc, compiling the translation units in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUTDIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUTDIR, "libpmmm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["pmmm.cu", "hier.cu", "sort.cu", "p2m_l2p.cu", "fft.cu", "m2l.cu", "green.cu", "pp.cu", "reduce.cu", "static_sort.cu", "batch.cu",
           "m2l_tc.cu", "fft_fused.cu", "mlp.cu", "surrogate.cu", "probe.cu"]
HEADERS = ["common.cuh", "harmonics.cuh", "translations.cuh", "fft.cuh", "internal.cuh", "binning.cuh",
           "m2l_table.cuh", "tcgen05.cuh", "plan.cuh"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                   "-I", INCLUDE, "-I", CSRC] + list(extra)


def _newest_dep() -> float:
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "pmmm.h"), os.path.abspath(__file__)]
    return max(os.path.getmtime(d) for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile every .cu to an object and link the shared library; returns its path."""
    os.makedirs(OUTDIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_dep():
        return LIB
    cc = nvcc()

    def one(src):
        obj = os.path.join(OUTDIR, os.path.splitext(src)[0] + ".o")
        cmd = [cc] + _flags(extra_flags) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    workers = min(len(SOURCES), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
