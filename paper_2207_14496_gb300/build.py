"""Build libfsl.so (the CUDA library behind include/fsl.h) for sm_103a.

Each translation unit is compiled by nvcc in parallel and linked into one
shared library inside the package (``_build/libfsl.so``).  Every unit is
compiled with ``-fmad=false`` (no multiply-add contraction): the FP64 kernels
then follow the source's operation order bit for bit, and a kernel body that
is compiled into more than one kernel (the single-domain and the batched
launch of a step kernel) gives the same bits in each, because the compiler
cannot contract a multiply and an add differently in the two.  The hot
16/32-bit collision spells out its fused multiply-adds explicitly.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libfsl.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

UNITS = {"fsl_api.cu": ["-fmad=false"], "fsl_noalloc.cu": ["-fmad=false"]}
for _p in ("fp64", "fp32", "fp16", "bf16"):
    for _q in (19, 27):
        UNITS[f"k_{_p}_q{_q}.cu"] = ["-fmad=false"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)
            if f.endswith((".cu", ".cuh", ".h"))] + [os.path.join(INCLUDE, "fsl.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", INCLUDE, "-I", CSRC, "-prec-div=true", "-prec-sqrt=true",
                     "-ftz=false"]
    if verbose:
        common += ["-Xptxas", "-v"]
    procs = []
    objs = []
    for unit, extra in UNITS.items():
        obj = os.path.join(OUT_DIR, unit.replace(".cu", f".{os.getpid()}.o"))
        objs.append(obj)
        cmd = [nvcc] + common + extra + ["-c", os.path.join(CSRC, unit), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT, text=True)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out)
        if p.returncode != 0:
            failed.append(" ".join(cmd))
    try:
        if failed:
            raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, check=True)
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
