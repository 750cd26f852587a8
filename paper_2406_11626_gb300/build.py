"""Builds the CCZ4 CUDA library for sm_103a, in tree.

Each translation unit under csrc/ is compiled by nvcc in parallel into
_build/, then linked into lib/libccz4_gb300.so. The FMA-throughput probe
under measure/ (used by bench.py to measure the FP64 and FP32 pipe rates)
is linked into a library of its own, lib/libccz4_peaks.so, so the product
library carries no measurement code. Rebuilds only what changed.
"""
import concurrent.futures as cf
import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
MEASURE = os.path.join(PKG, "measure")
LIB = os.path.join(LIBDIR, "libccz4_gb300.so")
PEAKS_LIB = os.path.join(LIBDIR, "libccz4_peaks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                     "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps(src):
    return [src] + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "ccz4.h")]


def _compile(src):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    log = obj + ".ptxas.log"
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in _deps(src)):
        return obj
    cmd = [_nvcc()] + NVCC_FLAGS + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    with open(log, "w") as f:
        f.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr[-6000:]))
    os.replace(obj + ".tmp", obj)
    return obj


def _link(lib, objs):
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [_nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
        subprocess.check_call(cmd)
        os.replace(tmp, lib)


def build(force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    if force:
        for f in glob.glob(os.path.join(BUILD, "*.o")):
            os.remove(f)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    probes = sorted(glob.glob(os.path.join(MEASURE, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs) + len(probes))) as ex:
        objs = list(ex.map(_compile, srcs + probes))
    _link(LIB, objs[:len(srcs)])
    _link(PEAKS_LIB, objs[len(srcs):])
    return LIB


if __name__ == "__main__":
    print(build())
