"""Compile the CUDA sources into the in-tree shared library libsipf.so.

One nvcc process per translation unit (run in parallel), then one link.
Target: sm_103a only.  particles.cu is compiled without FMA contraction so
that the count and scatter passes, which recompute the same particle push,
produce bit-identical positions from the same source expressions.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "libsipf.so")
BUILD = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-I", INC]
PER_FILE = {"particles.cu": ["-fmad=false"]}
SOURCES = ["api.cu", "particles.cu", "fft.cu", "fft_fused_p0.cu", "fft_fused_p1.cu",
           "fft_split_p0.cu", "fft_split_p1.cu", "fft_warp.cu", "noalloc.cu", "resample.cu", "server.cu",
           "smooth.cu"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(nvcc: str, src: str, extra: list[str], verbose_ptxas: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc, *ARCH, *COMMON, *PER_FILE.get(src, []), *extra, "-c",
           os.path.join(SRC, src), "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas:
        print(r.stderr)
    return obj


def build(extra: list[str] | None = None, verbose_ptxas: bool = False) -> str:
    """Build libsipf.so in the package directory and return its path."""
    extra = extra or []
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, extra, verbose_ptxas), SOURCES))
    tmp = OUT + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    import sys
    print(build(verbose_ptxas="-v" in sys.argv))
