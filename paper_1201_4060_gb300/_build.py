"""Build libbspline.so in-tree with nvcc for sm_103a (no cmake, parallel translation units)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libbspline.so")
# the checks build: every particle kernel with index checks that count failures in a status word
BUILD_CHECKS = os.path.join(BUILD, "checks")
LIB_CHECKS = os.path.join(BUILD_CHECKS, "libbspline_checks.so")
SOURCES = ["api.cu", "fft.cu", "particles.cu", "gather_f64_lo.cu", "gather_f64_hi.cu", "gather_f32_lo.cu",
           "gather_f32_hi.cu", "gather_bf16_lo.cu", "gather_bf16_hi.cu", "noalloc.cu", "adjoint_fft.cu",
           "adjoint_f32.cu", "adjoint_bf16.cu", "adjoint_f64.cu", "batch.cu", "batch_q_o2.cu", "batch_q_o3.cu",
           "batch_q_o4.cu", "batch_q_o5.cu", "batch_q_o6.cu", "batch_q_o7.cu", "batch_q_o8.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbspline.so")
    return exe


def _compile(src: str, extra: list[str], outdir: str = BUILD) -> str:
    obj = os.path.join(outdir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "bspline.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, checks: bool = False) -> str:
    """Compile every translation unit in parallel and link the shared library; return its path.
    checks=True builds the BSPLINE_CHECKS=1 variant (libbspline_checks.so) in its own folder."""
    lib = LIB_CHECKS if checks else LIB
    outdir = BUILD_CHECKS if checks else BUILD
    if not force and not _stale(lib):
        return lib
    os.makedirs(outdir, exist_ok=True)
    extra = list(extra or []) + (["-DBSPLINE_CHECKS=1"] if checks else [])
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, outdir), SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}", file=sys.stderr)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
