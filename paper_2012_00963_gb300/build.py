"""Build libpdv.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel into ``_build/`` and linked into
``paper_2012_00963_gb300/libpdv.so``. Only one ``-gencode`` target is built.
The debug library ``libpdv_debug.so`` is the same sources compiled with
``-DPDV_DEBUG`` (index checks in the kernels, path traces) into
``_build/debug/``; ``build(debug=True)`` makes it, ``build_all()`` makes both
in one parallel compile.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpdv.so")
LIB_DEBUG = os.path.join(PKG, "libpdv_debug.so")
SOURCES = ["tables.cu", "transport.cu", "spectra.cu", "stepping.cu", "api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code is compiled without FMA contraction (gcc contracts by default on
# Arm), so host-side floating point gives the same bits on x86 and Arm.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libpdv needs the CUDA toolkit to build")


def _deps() -> list:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    return files + [os.path.join(INCLUDE, "pdv.h"), os.path.abspath(__file__)]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _variants(debug_list, force):
    deps = _deps()
    out = []
    for debug in debug_list:
        lib = LIB_DEBUG if debug else LIB
        if force or _stale(lib, deps):
            out.append((debug, lib))
    return out


def _build(debug_list, force: bool = False, verbose: bool = False):
    todo = _variants(debug_list, force)
    if not todo:
        return
    cc = nvcc()

    def one(job):
        debug, src = job
        d = os.path.join(BUILD, "debug") if debug else BUILD
        os.makedirs(d, exist_ok=True)
        obj = os.path.join(d, os.path.splitext(src)[0] + ".o")
        cmd = [cc] + ARCH + FLAGS + (["-DPDV_DEBUG"] if debug else []) + \
            ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
        return debug, obj, r.stderr

    jobs = [(debug, src) for debug, _ in todo for src in SOURCES]
    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        results = list(ex.map(one, jobs))
    for debug, lib in todo:
        objs = [o for dbg, o, _ in results if dbg == debug]
        tmp = lib + ".tmp.%d" % os.getpid()
        r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True,
                           text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s" % r.stderr)
        os.replace(tmp, lib)
    if verbose:
        for _, _, err in results:
            print(err)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile (if needed) and return the path of libpdv.so (libpdv_debug.so
    with debug=True)."""
    _build([debug], force, verbose)
    return LIB_DEBUG if debug else LIB


def build_all(force: bool = False, verbose: bool = False) -> tuple:
    """Compile both libraries (release and debug) in one parallel pass."""
    _build([False, True], force, verbose)
    return LIB, LIB_DEBUG


if __name__ == "__main__":
    import sys
    print(build_all(force="--force" in sys.argv, verbose="-v" in sys.argv))
