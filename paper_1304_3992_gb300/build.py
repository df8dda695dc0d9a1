"""Builds libfx.so (the C-ABI CUDA library) in-tree for sm_103a.

Translation units compile in parallel (nvcc for .cu, g++ for .cpp) and link
with nvcc into paper_1304_3992_gb300/_build/libfx.so with the CUDA runtime
linked statically.  Rebuilds only when a source or header is newer than the
library.  Usage: python -m paper_1304_3992_gb300.build [--force] [--checked]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfx.so")
# the checked build: -DFX_CHECKED range-checks every kernel memory index
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libfx_checked.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home() -> str:
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(ROOT, "include", "fx.h"), os.path.abspath(__file__)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(src: str, extra: list[str], build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    if src.endswith(".cu"):
        extra = extra + [f"-D{k}={os.environ[k]}" for k in ("FX_FIRST_PASS_CTAS", "FX_WARPS_PER_CTA", "FX_BATCH_CTAS") if os.environ.get(k)]
        cmd = ["nvcc", ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr", *inc, *extra,
               "-c", src, "-o", obj]
    else:
        # the run-time compiler (fx_jit.cpp) reads the kernel headers from the
        # source tree and the toolkit's libnvrtc
        paths = [f'-DFX_SRC_DIR="{CSRC}"', f'-DFX_INC_DIR="{os.path.join(ROOT, "include")}"',
                 f'-DFX_CUDA_LIB_DIR="{os.path.join(_cuda_home(), "lib64")}"']
        extra = extra + [f"-D{k}={os.environ[k]}" for k in ("FX_FIRST_PASS_CTAS", "FX_WARPS_PER_CTA", "FX_BATCH_CTAS") if os.environ.get(k)]
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
               "-I" + os.path.join(_cuda_home(), "include"), *inc, *paths, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, checked: bool = False) -> str:
    """Compile every translation unit for sm_103a and link libfx.so (or, with
    checked=True, libfx_checked.so with -DFX_CHECKED); returns its path."""
    build_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    extra = list(extra or []) + (["-DFX_CHECKED"] if checked else [])
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), srcs))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = ["nvcc", ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}")
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv)
