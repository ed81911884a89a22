"""Compile the CUDA sources in ``csrc/`` into the in-tree ``_build/libwdlb.so``.

sm_103a only (``-gencode arch=compute_103a,code=sm_103a``); the translation
units compile in parallel.  nvcc cross-compiles without a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libwdlb.so")
# The checked build: every kernel index tested against its array (-DWDLB_CHECKED=1);
# an index outside it is reported through the status word instead of accessing memory.
LIB_CHECKED = os.path.join(OUT_DIR, "libwdlb_checked.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-fast-math",
         "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(ROOT, "include")]

# (object name, source, extra defines)
UNITS = [
    ("wdlb_api.o", "wdlb_api.cu", []),
    ("wdlb_launch_f64.o", "wdlb_launch.cu", ["-DWDLB_STORAGE=0"]),
    ("wdlb_launch_f32.o", "wdlb_launch.cu", ["-DWDLB_STORAGE=1"]),
    ("wdlb_launch_f32dw.o", "wdlb_launch.cu", ["-DWDLB_STORAGE=1", "-DWDLB_DW_COLLISION=1"]),
    ("wdlb_launch_f16.o", "wdlb_launch.cu", ["-DWDLB_STORAGE=2"]),
    ("wdlb_static.o", "wdlb_static.cu", []),
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(ROOT, "include", "wdlb.h"))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile the library (checked=True: the bounds-checked variant, a
    separate .so) and return its path; up to date sources are not rebuilt."""
    os.makedirs(OUT_DIR, exist_ok=True)
    lib = LIB_CHECKED if checked else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _sources_mtime():
        return lib
    cc = nvcc()
    tag = "_checked" if checked else ""
    defs = ["-DWDLB_CHECKED=1"] if checked else []

    def compile_unit(unit):
        obj, src, extra = unit
        obj = obj.replace(".o", tag + ".o")
        cmd = [cc, *ARCH, *FLAGS, *defs, *extra, "-c", os.path.join(CSRC, src), "-o", os.path.join(OUT_DIR, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[os.path.join(OUT_DIR, o) for o in objs], "-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
