"""Builds liborqa.so in-tree with nvcc for sm_103a (GB300).

The library is the CUDA translation units in ``csrc/`` plus the C ABI
header in ``include/``.  ``-fmad=false`` keeps every coefficient product and sum
separately rounded (the kernels also use explicit _rn intrinsics), so the
arithmetic matches a CPU evaluation of the per-gate update bit for bit.
"""
from __future__ import annotations

import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "liborqa.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cuh")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def translation_units():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def nvcc_cmd(out: str, extra=()):
    return ["nvcc", ARCH, "-O3", "-lineinfo", "-fmad=false", "-std=c++17",
            "-Xcompiler", "-fPIC", "-shared", "-I" + INCLUDE, *extra,
            "-o", out, *translation_units()]


def build(force: bool = False, verbose: bool = False) -> str:
    deps = sources() + [os.path.join(INCLUDE, "orqa.h"), __file__]
    if force or _stale(LIB, deps):
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = nvcc_cmd(tmp)
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
