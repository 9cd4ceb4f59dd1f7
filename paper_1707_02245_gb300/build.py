"""Builds the CUDA library libpat_pdhg.so in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into a shared library with
a plain C ABI (include/pat.h).  No PyTorch headers are involved.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIBNAME = "libpat_pdhg.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["geometry.cu", "projector.cu", "adjoint.cu", "pdhg.cu", "noalloc.cu", "conv.cu", "unet.cu", "preprocess.cu", "wavelet.cu", "dtcwt.cu"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build the library")
    return cand


def common_flags() -> list[str]:
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                   "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers += [os.path.join(INCLUDE, h) for h in ("pat.h", "pat_unet.h")]
    flags = common_flags() + (extra or [])
    # objects built with other flags (e.g. extra defines) are rebuilt
    stamp = os.path.join(BUILD, "flags.txt")
    same_flags = os.path.exists(stamp) and open(stamp).read() == " ".join(flags)
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if not same_flags or _stale(o, [s] + headers + [__file__]):
            jobs.append([nvcc()] + flags + ["-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        list(ex.map(run, jobs))
    if not same_flags:
        with open(stamp, "w") as fh:
            fh.write(" ".join(flags))
    out = lib_path()
    if jobs or _stale(out, objs):
        run([nvcc()] + ARCH + ["-shared", "-o", out] + objs + ["-lcudart"])
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
