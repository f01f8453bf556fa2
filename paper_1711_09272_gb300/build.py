"""Compiles the CUDA library libroeam.so in-tree for sm_103a (GB300).

The translation units (2D host ABI, FP32 and FP64 kernels, FP32 and FP64 ablation-variant
kernels; 3D host ABI, FP32 and FP64 3D kernels) compile in parallel with nvcc and link into
paper_1711_09272_gb300/_build/libroeam.so.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libroeam.so")
SOURCES = ["roeam_api.cu", "roeam_k32.cu", "roeam_k64.cu", "roeam_k32_abl.cu", "roeam_k64_abl.cu", "roeam3_api.cu",
           "roeam3_k32.cu", "roeam3_k64.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--prec-div=false", "--prec-sqrt=false",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]
# The 2D translation units write every fused multiply-add out explicitly and forbid the
# compiler from forming others, so that results are bit-identical across work-unit layouts
# (tile shapes, row slabs) and across the copies of an unrolled loop body.
EXACT_FMA = {"roeam_api.cu", "roeam_k32.cu", "roeam_k64.cu", "roeam_k32_abl.cu", "roeam_k64_abl.cu"}


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libroeam")
    return exe


DEBUG_DIR = os.path.join(HERE, "_build_debug")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", f) for f in
                                                              os.listdir(os.path.join(ROOT, "include"))] + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Builds libroeam.so if missing or older than its sources; returns its path. debug=True
    builds the bounds-checked library (-DROEAM_DEBUG: every state, mask and vertex access of the
    2D stage kernels is checked and reported as ROEAM_E_BOUNDS instead of faulting) into
    _build_debug/."""
    out_dir = DEBUG_DIR if debug else OUT_DIR
    lib_path = os.path.join(out_dir, "libroeam.so")
    if not force and not _stale(lib_path):
        return lib_path
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    objs = [os.path.join(out_dir, os.path.splitext(s)[0] + ".o") for s in SOURCES]

    def compile_one(k):
        extra = ["-fmad=false"] if SOURCES[k] in EXACT_FMA else []
        if debug:
            extra.append("-DROEAM_DEBUG")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, SOURCES[k]), "-o", objs[k]]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {SOURCES[k]}:\n{r.stderr}")
        return r.stderr

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        logs = list(ex.map(compile_one, range(len(SOURCES))))
    tmp = lib_path + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    if verbose:
        print("\n".join(logs))
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
