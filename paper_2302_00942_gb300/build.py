"""Build the RFD GB300 library in-tree: paper_2302_00942_gb300/librfd_gb300.so.

Every CUDA translation unit is compiled for sm_103a only
(-gencode arch=compute_103a,code=sm_103a), in parallel, and linked with the
static CUDA runtime so the library does not depend on which libcudart the
host process (e.g. PyTorch) has loaded.  Host-only code (step a1, the random
frequencies) is compiled by g++ without floating-point contraction so that its
FP64 arithmetic is exactly the rounded sequence its comments describe.

Usage:  python -m paper_2302_00942_gb300.build   (or build() from Python)
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
LIB = os.path.join(HERE, "librfd_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["tc_common.cu", "k_features.cu", "k_gram_simt.cu", "k_gram_tc.cu", "k_gram_pair.cu", "k_reduce_apply.cu", "k_fp64.cu",
              "k_ozaki.cu", "k_batch.cu", "k_apply_tc.cu", "rfd_batch.cu",
              "rfd_phi1.cu", "rfd_api.cu", "rfd_noalloc.cu", "rfd_server.cu", "rfd_barycenter.cu",
              "rfd_gw.cu", "rfd_eigen.cu"]
CPP_SOURCES = ["rfd_host.cpp"]


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)


def _stale(obj: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, jobs: int | None = None, extra_nvcc: list[str] | None = None) -> str:
    """Compile (incrementally) and link the library; return its path."""
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "rfd.h"))
    cmds, objs = [], []
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if _stale(o, [s] + headers):
            cmds.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
                         "-fvisibility=hidden", "--expt-relaxed-constexpr", *(extra_nvcc or []),
                         "-c", s, "-o", o])
    for src in CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if _stale(o, [s] + headers):
            cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fvisibility=hidden",
                         f"-I{cuda}/include", "-c", s, "-o", o])
    with cf.ThreadPoolExecutor(max_workers=jobs or min(8, os.cpu_count() or 4)) as ex:
        for cmd, fut in [(c, ex.submit(_run, c)) for c in cmds]:
            fut.result()
            if verbose:
                print(" ".join(cmd[:2]), cmd[-3], file=sys.stderr)
    if cmds or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        _run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
