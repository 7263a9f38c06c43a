"""Build libnrr.so (the CUDA hot path behind include/nrr.h) for sm_103a.

Each translation unit is compiled by nvcc in parallel into
``paper_2501_14030_gb300/_build/`` and linked into one shared library with the
CUDA runtime linked statically, so the library loads without torch.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libnrr.so")
# The NRR_DEBUG build (address checks in the stencil kernels' loads and
# stores) goes to its own folder and library name.
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libnrr_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-O2", "--expt-relaxed-constexpr",
              "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required")
    return path


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith(".cu"))


def _deps() -> list[str]:
    out = [os.path.join(ROOT, "include", f)
           for f in os.listdir(os.path.join(ROOT, "include"))]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC)
            if f.endswith((".cuh", ".h"))]
    return out


def _compile(src: str, extra: list[str], out_dir: str, defs: list[str]) -> str:
    obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
    newest_dep = max(os.path.getmtime(p) for p in _deps() + [src])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest_dep and not extra:
        return obj
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *defs, *extra, "-c", src, "-o", obj]
    subprocess.run(cmd, check=True)
    return obj


def build(verbose_ptxas: bool = False, force: bool = False,
          debug: bool = False) -> str:
    """Compile every CUDA source and link ``_build/libnrr.so`` (with
    debug=True: ``_build_debug/libnrr_debug.so``, compiled with
    -DNRR_DEBUG=1)."""
    out_dir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    defs = ["-DNRR_DEBUG=1"] if debug else []
    os.makedirs(out_dir, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    if force:
        for f in os.listdir(out_dir):
            if f.endswith(".o"):
                os.remove(os.path.join(out_dir, f))
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, out_dir, defs), srcs))
    if (not os.path.exists(lib) or force or extra
            or max(os.path.getmtime(o) for o in objs) > os.path.getmtime(lib)):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static",
               "-lrt", "-lpthread", "-ldl"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(verbose_ptxas="-v" in sys.argv, force="-f" in sys.argv,
                debug="--debug" in sys.argv))
