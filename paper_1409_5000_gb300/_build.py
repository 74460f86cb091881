"""In-tree build of the native libraries.

* ``_lib/libcb.so``      -- the C-ABI library (CUDA, sm_103a only), built
  with nvcc from ``csrc/*.cu``; one object per translation unit, compiled
  in parallel, then linked with ``-shared``.
* ``_lib/libcb_debug.so`` -- the same sources with ``-DCB_DEBUG``: every
  indexed access of the SpMV kernels checked on the device (a violation is
  counted and skipped, never trapped); loaded instead of libcb.so when the
  environment sets ``CB_DEBUG=1``.
* ``_lib/libcbsynth.so`` -- the seeded input generators (plain C, gcc).

Outputs are written to a temporary name and renamed, so that concurrent
builds (e.g. parallel test workers) never load a half-written library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["cb_api.cu", "cb_lanczos.cu", "cb_tridiag.cu", "cb_combine.cu", "cb_topk.cu",
              "cb_adjoint.cu", "cb_blocked.cu", "cb_generate.cu",
              "cb_subgraph.cu", "cb_restart.cu", "cb_twophase.cu"]


def cb_lib_path(debug: bool = False) -> str:
    return os.path.join(LIBDIR, "libcb_debug.so" if debug else "libcb.so")


def synth_lib_path() -> str:
    return os.path.join(LIBDIR, "libcbsynth.so")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _atomic_move(src: str, dst: str) -> None:
    os.replace(src, dst)


def build_synth() -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    out = synth_lib_path()
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=LIBDIR)
    os.close(fd)
    cc = shutil.which("gcc") or "cc"
    _run([cc, "-O2", "-fPIC", "-shared", "-std=c11", os.path.join(CSRC, "synth.c"), "-o", tmp,
          "-lm"])
    _atomic_move(tmp, out)
    return out


def _nvcc() -> str:
    p = os.path.join(CUDA_HOME, "bin", "nvcc")
    return p if os.path.exists(p) else (shutil.which("nvcc") or "nvcc")


def nvcc_flags(extra=()):
    return (["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler",
             "-fvisibility=hidden", "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
            + ARCH + list(extra))


def build_cb(verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    """Compile every CUDA translation unit for sm_103a and link libcb.so
    (libcb_debug.so with ``debug``)."""
    os.makedirs(LIBDIR, exist_ok=True)
    if debug:
        extra_flags = list(extra_flags) + ["-DCB_DEBUG"]
    objdir = tempfile.mkdtemp(prefix="obj_", dir=LIBDIR)
    try:
        nvcc = _nvcc()

        def comp(src):
            obj = os.path.join(objdir, src.replace(".cu", ".o"))
            cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + nvcc_flags(extra_flags)
            if verbose:
                cmd += ["-Xptxas", "-v"]
            return obj, _run(cmd)

        with ThreadPoolExecutor(len(CU_SOURCES)) as ex:
            results = list(ex.map(comp, CU_SOURCES))
        if verbose:
            for _, log in results:
                print(log)
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=LIBDIR)
        os.close(fd)
        _run([nvcc, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH
             + ["-Xcompiler", "-fPIC", "-cudart", "static"])
        _atomic_move(tmp, cb_lib_path(debug))
    finally:
        shutil.rmtree(objdir, ignore_errors=True)
    return cb_lib_path(debug)


def build_all(verbose: bool = False) -> None:
    build_synth()
    build_cb(verbose=verbose)
    build_cb(debug=True)
