"""Builds libmgdarcy.so in-tree for sm_103a (nvcc, parallel translation units).

    python -m paper_1602_04858_gb300.build [--verbose]

Object files go to paper_1602_04858_gb300/_build/, the library to
paper_1602_04858_gb300/libmgdarcy.so.  A unit is recompiled when its source
or any header in csrc/ is newer than its object.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmgdarcy.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
                  "-I" + CSRC, "-I" + INCLUDE, "--expt-relaxed-constexpr"]

UNITS = [
    ("kinst.cu", "k20.o", ["-DMG_D=2", "-DMG_K=0"]),
    ("kinst.cu", "k21.o", ["-DMG_D=2", "-DMG_K=1"]),
    ("kinst.cu", "k22.o", ["-DMG_D=2", "-DMG_K=2"]),
    ("kinst.cu", "k30.o", ["-DMG_D=3", "-DMG_K=0"]),
    ("generic.cu", "generic.o", []),
    ("api.cu", "api.o", []),
    ("noalloc.cu", "noalloc.o", []),
    ("peaks.cu", "peaks.o", []),
    ("cnn.cu", "cnn.o", []),
    ("tables.cpp", "tables.o", ["-x", "cu"]),
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _newest_header() -> float:
    t = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".h", ".cuh")):
                t = max(t, os.path.getmtime(os.path.join(d, f)))
    return t


def build(verbose: bool = False, extra=None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    hdr = _newest_header()
    cmds = []
    objs = []
    for src, obj, defs in UNITS:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, obj)
        objs.append(o)
        if os.path.exists(o) and os.path.getmtime(o) >= max(os.path.getmtime(s), hdr):
            continue
        cmds.append([nvcc()] + NVFLAGS + list(extra or []) + defs + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=min(8, max(1, len(cmds)))) as ex:
        for cmd, r in ex.map(run, cmds):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed for " + cmd[-3])
    if cmds or not os.path.exists(LIB):
        link = [nvcc()] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart"]
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(link) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="--verbose" in sys.argv))
