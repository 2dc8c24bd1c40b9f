"""Builds libgrom.so (the CUDA library behind include/grom.h) for sm_103a.

Each translation unit is compiled by nvcc in parallel and linked into a
shared library inside the package directory.  No CMake, no torch extension
machinery: the library has a plain C ABI.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgrom.so")

SOURCES = [
    "api.cu",
    "k_convert.cu",
    "k_step.cu",
    "k_svd.cu",
    "als.cu",
    "k3_cp.cu",
    "k3_gemm.cu",
    "k3_ds.cu",
    "k3_oz.cu",
    "k3_persistent.cu",
    "k1_plan.cu",
    "k1_f64.cu",
    "k1_f32x2.cu",
    "k1_f32.cu",
    "k1_bf16.cu",
    "k1_static.cu",
    "k1p_f64.cu",
    "k1p_f32x2.cu",
    "k1p_f32.cu",
    "k1p_bf16.cu",
    "k1pp_f64.cu",
    "k1pp_f32x2.cu",
    "k1pp_f32.cu",
    "k1pp_bf16.cu",
    "k2_tc.cu",
    "k2p_tc.cu",
    "k3t_tc.cu",
    "serve.cu",
]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "grom.h"))
    files.append(os.path.abspath(__file__))
    return files


def stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force=False, verbose=False, jobs=None):
    """Compile every CUDA source and link libgrom.so; returns its path."""
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + NVCC_FLAGS + ["-I" + os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj

    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with concurrent.futures.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
