"""Build libaxpic.so in-tree with nvcc for sm_103a (no CMake, no torch
extension: the library's ABI is plain C). Translation units compile in
parallel, then link into paper_2604_24627_gb300/libaxpic.so."""
import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libaxpic.so")
SOURCES = ["api.cu", "step.cu", "misc.cu", "mlp.cu", "sr.cu", "stream.cu", "merge.cu", "tables.cpp", "surrogate.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", os.path.join(ROOT, "include")]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src, defines=(), tag=""):
    obj = os.path.join(BUILD, tag + os.path.basename(src) + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + ["-D" + d for d in defines] + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj


def build(verbose=False, defines=(), out=None):
    """Compile and link; `defines` (NAME=VALUE strings) and `out` select a
    variant build (launch-shape tuning), the default is the package library."""
    os.makedirs(BUILD, exist_ok=True)
    tag = "_".join(d.replace("=", "") for d in defines) + "_" if defines else ""
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, defines, tag), SOURCES))
    lib = out or LIB
    tmp = lib + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    if verbose:
        print("built", lib)
    return lib


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
