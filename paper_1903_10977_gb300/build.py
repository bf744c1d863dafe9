"""Builds libimgm.so in the package directory (nvcc for sm_103a, g++ for the host setup).

Run as ``python paper_1903_10977_gb300/build.py`` or through ``__graft_entry__.build()``.  Translation
units compile in parallel; nothing is rebuilt when the library is newer than every
source file.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libimgm.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cpp", ".cuh", ".hpp"))] + [os.path.join(INCLUDE, "imgm.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    cxx = shutil.which("g++") or "g++"
    tmp = tempfile.mkdtemp(prefix="imgm_build_")
    jobs = []
    objs = []
    common_nv = [nvcc, ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp", "-I", INCLUDE]
    for f in sorted(x for x in os.listdir(CSRC) if x.endswith(".cu")):
        o = os.path.join(tmp, f + ".o")
        objs.append(o)
        jobs.append(common_nv + ["-c", os.path.join(CSRC, f), "-o", o])
    o = os.path.join(tmp, "setup.o")
    objs.append(o)
    jobs.append([cxx, "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-I", INCLUDE, "-c",
                 os.path.join(CSRC, "setup.cpp"), "-o", o])
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for j in jobs]
    errors = []
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        if verbose and out:
            print(out)
        if p.returncode != 0:
            errors.append(" ".join(j) + "\n" + out)
    if errors:
        raise RuntimeError("libimgm build failed:\n" + "\n".join(errors))
    link = [nvcc, ARCH, "-shared", "-o", LIB + ".tmp"] + objs + ["-lgomp", "-lcudart"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("libimgm link failed:\n" + " ".join(link) + "\n" + r.stdout)
    os.replace(LIB + ".tmp", LIB)
    shutil.rmtree(tmp, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
