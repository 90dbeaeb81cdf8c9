"""Build libhemelb_gb300.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in its own nvcc process (in parallel), then
one nvcc call links the shared library.  Nothing is installed: the library
lands in ``paper_1906_11925_gb300/_build/``.  ``ptxas -v`` resource usage is
kept in ``_build/ptxas.log``.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhemelb_gb300.so")
# the same library with range-checked table loads in the step kernels
# (HGB_CHECK_TABLE=1); loaded instead of LIB when HEMELB_GB300_CHECKED=1
CHECKED_LIB = os.path.join(BUILD, "libhemelb_gb300_checked.so")
CHECKED_SOURCE = "lbm_step.cu"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhemelb_gb300")
    return cand


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(ROOT, "include", "lbm.h"), os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(CHECKED_LIB):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(CHECKED_LIB))
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp,-fvisibility=hidden",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC] + ARCH
    procs = []
    objs = []
    checked_objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [nvcc, "-c", src, "-o", obj] + common
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                            text=True)))
        if os.path.basename(src) == CHECKED_SOURCE:
            cobj = os.path.join(BUILD, os.path.basename(src) + ".checked.o")
            checked_objs.append(cobj)
            ccmd = [nvcc, "-c", src, "-o", cobj, "-DHGB_CHECK_TABLE=1"] + common
            procs.append((src + " (checked)", subprocess.Popen(ccmd, stdout=subprocess.PIPE,
                                                               stderr=subprocess.STDOUT, text=True)))
        else:
            checked_objs.append(obj)
    logs = []
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        logs.append("== %s\n%s" % (os.path.basename(src), out))
        if p.returncode != 0:
            failed.append(src)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
        fh.write("\n".join(logs))
    if failed:
        sys.stderr.write("\n".join(logs))
        raise RuntimeError("nvcc failed for %s" % ", ".join(os.path.basename(f) for f in failed))
    for lib, lib_objs in ((CHECKED_LIB, checked_objs), (LIB, objs)):
        tmp = lib + ".tmp"
        cmd = [nvcc, "-shared", "-o", tmp] + lib_objs + ARCH + ["-Xcompiler", "-fopenmp"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout)
            raise RuntimeError("linking %s failed" % os.path.basename(lib))
        os.replace(tmp, lib)
    if verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
