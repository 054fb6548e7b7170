"""In-tree build of libgrmhd.so for sm_103a (nvcc + g++, translation units in parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgrmhd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["kernels_point.cu", "kernels_deriv.cu", "kernels_eo.cu", "kernels_tc.cu", "kernels_fx.cu", "api.cu",
      "noalloc.cu", "kernels_xcts.cu"]
CPP = ["host_ops.cpp", "host_eig.cpp"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgrmhd.so")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose: bool = False) -> str:
    """Compile every translation unit and link the shared library; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for f in CU:
        jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xptxas", "-v", "-c", os.path.join(CSRC, f), "-o",
                     os.path.join(BUILD, f + ".o")])
    for f in CPP:
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-I/usr/local/cuda/include", "-c",
                     os.path.join(CSRC, f), "-o", os.path.join(BUILD, f + ".o")])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    objs = [os.path.join(BUILD, f + ".o") for f in CU + CPP]
    tmp = LIB + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-ldl"])
    os.replace(tmp, LIB)
    if verbose:
        for lg in logs:
            print(lg)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
        fh.write("\n".join(logs))
    return LIB
