"""In-tree build of the le_mc CUDA library (``libLeMC.so``) for sm_103a.

Each translation unit is compiled by nvcc in parallel into ``_build/`` and
linked (CUDA runtime statically) into ``paper_1206_3316_gb300/libLeMC.so``.
Nothing is installed; the shared object sits next to the Python binding.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
OBJ = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libLeMC.so")
LIB_DEBUG = os.path.join(PKG, "libLeMC_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# FP32 trajectories use approximate division / square root and flush denormals;
# FP64 arithmetic is unaffected by these flags.
CUFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I" + INC,
                  "-ftz=true", "-prec-div=false", "-prec-sqrt=false"]
# (source, object name, extra flags): the trace kernels' source is compiled
# once per trajectory precision
SOURCES = [("trace_launch.cu", "trace_f32", ["-DLEMC_PREC_BITS=32"]),
           ("trace_launch.cu", "trace_f64", ["-DLEMC_PREC_BITS=64"]),
           ("le_mc_api.cu", "le_mc_api", []), ("le_mc_batch.cu", "le_mc_batch", []),
           ("le_mc_server.cu", "le_mc_server", []), ("le_mc_noalloc.cu", "le_mc_noalloc", []),
           ("le_mc_diag.cu", "le_mc_diag", []), ("serve_kernel.cu", "serve_kernel", []),
           ("le_mc_host.cpp", "le_mc_host", [])]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the le_mc library needs the CUDA toolkit to build")
    return exe


def _newest_input():
    paths = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(INC, "le_mc.h"), __file__]
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build libLeMC.so, or with ``debug`` the checking variant
    libLeMC_debug.so (-DLEMC_DEBUG: out-of-range kernel indices are reported
    in the run's device flags instead of being trusted)."""
    lib = LIB_DEBUG if debug else LIB
    obj_dir = os.path.join(OBJ, "debug") if debug else OBJ
    flags = CUFLAGS + (["-DLEMC_DEBUG"] if debug else [])
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    os.makedirs(obj_dir, exist_ok=True)
    exe = nvcc()

    def compile_one(item):
        src, name, extra = item
        obj = os.path.join(obj_dir, name + ".o")
        cmd = [exe] + flags + extra + ["-c", os.path.join(SRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stderr}")
        if verbose:
            print(res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    res = subprocess.run([exe] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, debug="--debug" in sys.argv))
