"""In-tree build of the native parts of the package.

Compiles the CUDA library (``libsimlod.so``, sm_103a only) and the seeded
input generator (``synth/libsynth.so``). Both land next to their sources and
are rebuilt only when a source or header is newer than the built file.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
REPO_DIR = os.path.dirname(PKG_DIR)
INCLUDE_DIR = os.path.join(REPO_DIR, "include")
CSRC_DIR = os.path.join(PKG_DIR, "csrc")
LIB_PATH = os.path.join(PKG_DIR, "libsimlod.so")
SYNTH_DIR = os.path.join(PKG_DIR, "synth")
SYNTH_LIB = os.path.join(SYNTH_DIR, "libsynth.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _run(cmd: list[str]) -> None:
    proc = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if proc.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + proc.stdout)


def library_sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC_DIR, "*.cu")))


def library_headers() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC_DIR, "*.cuh")) +
                  glob.glob(os.path.join(INCLUDE_DIR, "*.h")))


def library_command(out: str = LIB_PATH, extra: list[str] | None = None) -> list[str]:
    # -dlcm=cg: plain global loads are served by the coherent L2, not the
    # per-SM L1, because the persistent kernel re-reads node tables, split
    # lists and grids that other blocks rewrote after a grid barrier (L1s are
    # not coherent with each other within one grid). Batch points are read
    # with __ldcg too: a merged update reads them from a staging buffer that
    # the same launch has just written.
    return ([_nvcc(), *ARCH_FLAGS, "-O3", "-lineinfo", "-std=c++17", "-shared",
             "-Xptxas", "-dlcm=cg",
             "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
             "-I", INCLUDE_DIR, "-I", CSRC_DIR]
            + (extra or []) + library_sources() + ["-o", out])


def build_library(force: bool = False) -> str:
    srcs = library_sources() + library_headers() + [os.path.abspath(__file__)]
    if force or _stale(LIB_PATH, srcs):
        tmp = LIB_PATH + ".tmp"
        _run(library_command(tmp))
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def build_synth(force: bool = False) -> str:
    src = os.path.join(SYNTH_DIR, "synth.c")
    if force or _stale(SYNTH_LIB, [src]):
        tmp = SYNTH_LIB + ".tmp"
        _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", src, "-o", tmp, "-lm"])
        os.replace(tmp, SYNTH_LIB)
    return SYNTH_LIB


def build_all(force: bool = False) -> None:
    build_synth(force)
    build_library(force)
