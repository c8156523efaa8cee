"""Build libgvx (the CUDA kernels and the C ABI) for sm_103a, in-tree.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel, then linked into
``_build/libgvx_<machine>.so`` (the machine suffix keeps an x86 cross-build and an aarch64 build
of the same tree apart).  Usage: ``python -m paper_2312_02756_gb300.build [--force] [--ptxas-v]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
# GVX_DEBUG_BOUNDS=1 in the environment builds and loads a separate variant with the explicit
# index checks of the jagged kernels compiled in (csrc/common.cuh, GVX_IN_BOUNDS).
DEBUG_BOUNDS = os.environ.get("GVX_DEBUG_BOUNDS", "") == "1"
_VARIANT = "dbg_" if DEBUG_BOUNDS else ""
LIB_PATH = os.path.join(BUILD, "libgvx_%s%s.so" % (_VARIANT, platform.machine()))
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
              "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC, "-I" + BUILD]
TABLES = os.path.join(BUILD, "gvx_tables.inc")


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the gvx CUDA library cannot be built")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "gvx.h"))
    files.append(os.path.abspath(__file__))
    files.append(os.path.join(PKG, "gen_tables.py"))
    files.append(TABLES)
    return files


def generate_tables(path: str = None) -> str:
    """Write the elementary-function tables the float-float kernels include."""
    from . import gen_tables
    return gen_tables.write(path or TABLES)


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, ptxas_verbose: bool = False, quiet: bool = True) -> str:
    """Compile (if stale) and return the path of the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    generate_tables()
    deps = _deps()
    if not force and not _stale(LIB_PATH, deps):
        return LIB_PATH
    exe = nvcc()
    srcs = _sources()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + "_%s%s.o" % (_VARIANT, platform.machine()))
            for s in srcs]
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []
    if DEBUG_BOUNDS:
        extra.append("-DGVX_DEBUG_BOUNDS")

    def compile_one(pair):
        src, obj = pair
        cmd = [exe, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if ptxas_verbose or not quiet:
        for s, log in zip(srcs, logs):
            if log.strip():
                sys.stderr.write("== %s\n%s" % (os.path.basename(s), log))
    tmp = LIB_PATH + ".tmp"
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    if __package__ in (None, ""):
        sys.path.insert(0, ROOT)
        from paper_2312_02756_gb300 import build as _self
        sys.exit(print(_self.build(force="--force" in sys.argv,
                                   ptxas_verbose="--ptxas-v" in sys.argv, quiet=False)))
    print(build(force="--force" in sys.argv, ptxas_verbose="--ptxas-v" in sys.argv,
                quiet=False))
