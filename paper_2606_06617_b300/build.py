"""Builds libpswf_lr.so in-tree with nvcc for sm_103a.

Usage: ``python -m paper_2606_06617_b300.build [-v]`` (or
``__graft_entry__.build()``).  Translation units are compiled in parallel into
``_build/`` and linked into ``paper_2606_06617_b300/libpswf_lr.so``; the
library links the CUDA runtime and cuFFT dynamically.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libpswf_lr.so")
# the same library with non-trapping bounds checks in the kernels
# (-DPSWF_BOUNDS_CHECK; a failed check is reported by pswf_sync as
# PSWF_EBOUNDS): for tests, not for timing
LIB_CHECKED = os.path.join(HERE, "libpswf_lr_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, object, extra flags)
UNITS = [
    ("api.cu", "api.o", []),
    ("launch.cu", "launch_f32.o", ["-DPSWF_REAL=float"]),
    ("launch.cu", "launch_f64.o", ["-DPSWF_REAL=double"]),
    ("planner.cpp", "planner.o", []),
    ("server.cu", "server.o", []),
    ("fft_x.cu", "fft_x.o", []),
    ("realspace.cu", "realspace.o", []),
]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "pswf_lr.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(verbose: bool = False, ptxas_verbose: bool = False, force: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    if os.path.exists(lib) and not (force or ptxas_verbose) and os.path.getmtime(lib) >= _newest_input():
        return lib
    os.makedirs(bdir, exist_ok=True)
    nvcc = nvcc_path()
    common = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I", INCLUDE, "-I", CSRC] + (["-DPSWF_BOUNDS_CHECK"] if checked else [])
    if ptxas_verbose:
        common.append("-Xptxas=-v")
    procs = []
    for src, obj, extra in UNITS:
        cmd = [nvcc, *common, *extra, "-c", os.path.join(CSRC, src), "-o", os.path.join(bdir, obj)]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    failed = False
    for cmd, pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            failed = True
            sys.stderr.write(" ".join(cmd) + "\n" + out + err)
        elif verbose or ptxas_verbose:
            sys.stderr.write(err)
    if failed:
        raise RuntimeError("nvcc failed building libpswf_lr.so")
    link = [nvcc, *ARCH, "-shared", "-o", lib + ".tmp", *[os.path.join(bdir, u[1]) for u in UNITS], "-lcufft"]
    res = subprocess.run(link, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc link of libpswf_lr.so failed")
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, ptxas_verbose="--ptxas" in sys.argv, force="-f" in sys.argv,
                checked="--checked" in sys.argv))
