"""Builds the CUDA library ``libmhdgpu.so`` in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel; the FP64 parity kernels and the
level operations use --fmad=false (bit-reproducible), the contracted FP64
kernels --fmad=true, the FP32 kernels --fmad=true --use_fast_math.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libmhdgpu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
          "-I" + SRC]
UNITS = {
    "capi.cu": [],
    "level_ops.cu": ["--fmad=false"],
    "advance_f64.cu": ["--fmad=false"],
    "advance_f64c.cu": ["--fmad=true"],
    "advance_f32.cu": ["--fmad=true", "--use_fast_math"],
    "noalloc.cu": ["--fmad=false"],
    "amr_ops.cu": ["--fmad=false"],
    "tree.cu": [],
    "hilbert.cu": ["--fmad=false", "-Xcompiler", "-ffp-contract=off"],
    "cluster.cu": ["-Xcompiler", "-ffp-contract=off"],
    "probe.cu": ["--fmad=true"],
    "regrid.cu": ["--fmad=false"],
}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _inputs():
    return [os.path.join(SRC, f) for f in sorted(os.listdir(SRC))] + [os.path.join(ROOT, "include", "mhd_gpu.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()

    def one(unit):
        obj = os.path.join(OUT, unit.replace(".cu", ".o"))
        cmd = [nvcc] + ARCH + COMMON + UNITS[unit] + (["-Xptxas", "-v"] if ptxas_v else []) + [
            "-c", os.path.join(SRC, unit), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (unit, " ".join(cmd), r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        res = list(ex.map(one, list(UNITS)))
    if verbose or ptxas_v:
        for _, err in res:
            if err:
                print(err)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in res]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    build(force=True, verbose=True, ptxas_v="-v" in sys.argv)
    print(LIB)
