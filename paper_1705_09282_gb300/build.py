"""Builds the in-tree shared library libigamg.so for sm_103a (nvcc + g++, no cmake).

    python -m paper_1705_09282_gb300.build
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libigamg.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -ffp-contract=off for host code: the host set-up rounds the same way on x86-64 and aarch64
# (gcc contracts a*b+c into fused multiply-adds on aarch64 by default); device code keeps FMA
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC] + ARCH
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    if "-c" in cmd:                                   # remember how the object was built
        with open(cmd[cmd.index("-o") + 1] + ".cmd", "w") as fh:
            fh.write(" ".join(cmd))
    return r.stdout


def _stale(src, obj, cmd):
    """An object is rebuilt when it is missing, older than its source or any header of the
    package, or was built with another command line (kept beside it as <obj>.cmd)."""
    stamp = obj + ".cmd"
    if not (os.path.exists(obj) and os.path.exists(stamp)):
        return True
    if open(stamp).read() != " ".join(cmd):
        return True
    heads = [os.path.join(d, f) for d in (CSRC, INCLUDE) for f in os.listdir(d)
             if f.endswith((".h", ".cuh"))]
    newest = max(os.path.getmtime(x) for x in [src] + heads)
    return os.path.getmtime(obj) < newest


def build(verbose=False, extra_nvcc=()):
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cu, cpp = _sources()
    jobs, objs = [], []
    for f in cu:
        o = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, f), "-o", o] + NVCC_FLAGS + list(extra_nvcc)
        if _stale(os.path.join(CSRC, f), o, cmd):
            jobs.append(cmd)
        objs.append(o)
    for f in cpp:
        o = os.path.join(BUILD, f + ".o")
        cmd = ["g++", "-c", os.path.join(CSRC, f), "-o", o] + CXX_FLAGS
        if _stale(os.path.join(CSRC, f), o, cmd):
            jobs.append(cmd)
        objs.append(o)
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs) or 1, os.cpu_count() or 4))) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = LIB + ".tmp"
    _run([nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart_static", "-Xcompiler", "-pthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv,
                extra_nvcc=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
