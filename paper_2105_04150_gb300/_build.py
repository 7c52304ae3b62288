"""Build the in-tree CUDA library ``_libpd.so`` for sm_103a.

Each translation unit is compiled in parallel (nvcc for .cu, g++ for .cpp),
then linked with nvcc into one shared library next to this file.  Host code
is compiled with ``-ffp-contract=off`` so that family search and notch tests
give the same answers on x86-64 and aarch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "_libpd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# per-file device flags: the FP32-bulk kernel uses approximate rsqrt/division
FAST_MATH = {"pd_step_f32.cu", "pd_step_f32_soft.cu", "pd_step_f32_ext.cu",
             "pd_step_f32_osb.cu", "pd_step_f32_lat.cu", "pd_step_f32_lat_batch.cu",
             "pd_step_f32_lat_r80.cu", "pd_step_f32_lat_batch_r80.cu",
             "pd_step_f32_lat_osb.cu", "pd_step_f32_lat_tma.cu"}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _cuda_home() -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(_nvcc())))


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) +
                  glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def _compile(src: str) -> str:
    name = os.path.basename(src)
    obj = os.path.join(OUT, name + ".o")
    if src.endswith(".cu"):
        cmd = [_nvcc(), "-c", src, "-o", obj, "-O3", "-std=c++17", "-lineinfo", *ARCH,
               "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off", "-Xptxas", "-v"]
        if name in FAST_MATH:
            cmd.append("--use_fast_math")
    else:
        cmd = ["g++", "-c", src, "-o", obj, "-O3", "-std=c++17", "-fPIC", "-fopenmp",
               "-ffp-contract=off", "-I", os.path.join(_cuda_home(), "include")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    with open(obj + ".log", "w") as f:
        f.write(r.stdout + r.stderr)
    return obj


def build(force: bool = False) -> str:
    srcs = _sources()
    newest = max(os.path.getmtime(p) for p in srcs + _headers() + [__file__])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(OUT, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(_compile, srcs))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [_nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def ptxas_report() -> str:
    """Register / spill / shared-memory lines of the last build (``-Xptxas -v``)."""
    out = []
    for log in sorted(glob.glob(os.path.join(OUT, "*.cu.o.log"))):
        for line in open(log):
            if "registers" in line or "spill" in line or "Compiling entry" in line:
                out.append(line.rstrip())
    return "\n".join(out)


if __name__ == "__main__":
    print(build(force=True))
    print(ptxas_report())
