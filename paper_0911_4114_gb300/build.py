"""Builds the in-tree shared library libhfmm.so (CUDA for sm_103a + host C++).

Host C++ (planner, special functions) is compiled by g++ with -ffp-contract=off so the
tree arithmetic rounds exactly as written; the CUDA translation unit by nvcc for
sm_103a only.  The three compiles run in parallel.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhfmm.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhfmm.so")
    return cand


def build(verbose=False, extra_nvcc=()):
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    host = ["-O2", "-fPIC", "-fopenmp", "-ffp-contract=off", "-std=c++17"]
    jobs = []
    objs = []
    for src in ("planner.cpp", "special.cpp"):
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        jobs.append(["g++", *host, "-c", os.path.join(CSRC, src), "-o", obj])
    for src in ("api.cu", "noalloc.cu", "tables.cu"):
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        jobs.append([nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     *extra_nvcc, "-c", os.path.join(CSRC, src), "-o", obj])
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for j in jobs]
    failed = []
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(" ".join(j))
    if failed:
        raise RuntimeError("compile failed:\n" + "\n".join(failed))
    tmp = LIB + ".tmp"
    link = [nvcc, ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        sys.stdout.write(r.stdout.decode(errors="replace"))
        raise RuntimeError("link failed: " + " ".join(link))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
