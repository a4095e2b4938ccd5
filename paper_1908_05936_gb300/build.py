"""Build libhc.so in-tree: every CUDA translation unit compiled for sm_103a in
parallel with nvcc, then linked into one shared library.  The user kernels of
examples/ (written against the public headers only) become
libhc_examples.so.

    python -m paper_1908_05936_gb300.build
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhc.so")
EXAMPLES_SRC = os.path.join(HERE, "examples", "device_api.cu")
EXAMPLES_LIB = os.path.join(HERE, "libhc_examples.so")
DEBUG_LIB = os.path.join(HERE, "libhc_debug.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         f"-I{os.path.join(ROOT, 'include')}"]

SOURCES = ["hc_api.cu", "hc_batch.cu", "hc_probe.cu", "hc_select.cu", "hc_ordered.cu", "hc_mixed.cu", "hc_serve.cu", "hc_kind_set_u32.cu", "hc_kind_set_u64.cu",
           "hc_kind_map_i64_i32.cu", "hc_kind_map_u64_u64.cu"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhc.so")
    return p


def _deps() -> list[str]:
    inc = os.path.join(ROOT, "include")
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(inc, f) for f in os.listdir(inc)]


def _example_deps() -> list[str]:
    inc = os.path.join(ROOT, "include")
    return [EXAMPLES_SRC, os.path.join(inc, "hc.h"), os.path.join(inc, "hc_device.cuh"),
            os.path.join(inc, "hc_core.cuh")]


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = _example_deps() if lib == EXAMPLES_LIB else _deps()
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra: list[str], build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    return obj


def build_examples(force: bool = False, verbose: bool = False) -> str:
    """Compile libhc_examples.so (the device-API user kernels); returns its path."""
    if not force and not stale(EXAMPLES_LIB):
        return EXAMPLES_LIB
    tmp = EXAMPLES_LIB + ".tmp"
    cmd = [nvcc(), *ARCH, *FLAGS, "-shared", EXAMPLES_SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {EXAMPLES_SRC}:\n{r.stderr}")
    os.replace(tmp, EXAMPLES_LIB)
    if verbose:
        print(f"built {EXAMPLES_LIB}")
    return EXAMPLES_LIB


def build(force: bool = False, extra: list[str] | None = None, verbose: bool = False, lib: str = LIB) -> str:
    """Compile and link libhc.so (or `lib`, with `extra` nvcc flags) next to
    this file; returns its path."""
    if not force and not stale(lib):
        return lib
    build_dir = BUILD if lib == LIB else os.path.join(BUILD, os.path.splitext(os.path.basename(lib))[0])
    os.makedirs(build_dir, exist_ok=True)
    extra = extra or []
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}")
    return lib


def build_debug(force: bool = False, verbose: bool = False) -> str:
    """libhc_debug.so: the same library with the debug bounds checks
    (-DHC_DEBUG): every bucket and slot index is checked against the table and
    every key range against its call; a violation sets error bit 4 of the
    table header (hc_stats, hc_status) instead of faulting."""
    return build(force=force, extra=["-DHC_DEBUG"], verbose=verbose, lib=DEBUG_LIB)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    build_examples(force="--force" in sys.argv, verbose=True)
    if "--debug" in sys.argv:
        build_debug(force="--force" in sys.argv, verbose=True)
