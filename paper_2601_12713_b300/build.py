"""Builds libodp.so, the OMPT tool libodp_ompt.so (and the synthetic-input
libraries) in-tree with nvcc for sm_103a.  Run
``python -m paper_2601_12713_b300.build``."""

from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libodp.so")
OMPT_SRC = os.path.join(PKG, "ompt", "ompt_tool.cpp")
OMPT_LIB = os.path.join(PKG, "libodp_ompt.so")
SYNTH_SRC = os.path.join(ROOT, "synth", "gen.cu")
SYNTH_LIB = os.path.join(ROOT, "synth", "libsynth.so")
LOADGEN_SRC = os.path.join(ROOT, "synth", "loadgen.cpp")
LOADGEN_LIB = os.path.join(ROOT, "synth", "libsynth_load.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
         "--expt-relaxed-constexpr", "-Xptxas", "-v"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(INCLUDE, "odp.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _nvcc(out, srcs, extra=(), log=None):
    tmp = out + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, *FLAGS, "-I", INCLUDE, "-I", CSRC, *extra, "-o", tmp, *srcs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if log is not None:
        with open(log, "w") as f:
            f.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError(f"nvcc failed for {out}")
    os.replace(tmp, out)


def build(force: bool = False, verbose: bool = False) -> str:
    if force or _stale(LIB, _deps()):
        _nvcc(LIB, _sources(), log=os.path.join(PKG, "build.log"))
        if verbose:
            print(open(os.path.join(PKG, "build.log")).read())
    if force or _stale(OMPT_LIB, [OMPT_SRC, LIB, os.path.join(INCLUDE, "odp.h"),
                                  os.path.join(INCLUDE, "odp_ompt.h")]):
        # host code only; links libodp.so from the same directory
        tmp = OMPT_LIB + f".tmp{os.getpid()}"
        cmd = [NVCC, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-I", INCLUDE,
               "-o", tmp, OMPT_SRC, "-L", PKG, "-lodp", "-Xlinker", "-rpath=$ORIGIN"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            sys.stderr.write(res.stdout + res.stderr)
            raise RuntimeError("nvcc failed for the OMPT tool")
        os.replace(tmp, OMPT_LIB)
    if force or _stale(SYNTH_LIB, [SYNTH_SRC]):
        _nvcc(SYNTH_LIB, [SYNTH_SRC])
    if force or _stale(LOADGEN_LIB, [LOADGEN_SRC]):
        tmp = LOADGEN_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o",
                               tmp, LOADGEN_SRC])
        os.replace(tmp, LOADGEN_LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
