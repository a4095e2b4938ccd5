"""GPU versions of the splitmix64 streams (gen.cu), for workloads too large to
draw quickly with numpy.  Each function returns a CUDA tensor whose bits equal
the numpy generator's output (checked by a GPU test)."""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

from . import splitmix as sm

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gen.cu")
LIB = os.path.join(HERE, "_build", "libhcgen.so")
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC",
                    SRC, "-o", LIB], check=True)
    return LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        ll, ull, vp = ctypes.c_longlong, ctypes.c_ulonglong, ctypes.c_void_p
        lib.hcgen_stream.argtypes = [vp, ll, ll, ull, ctypes.c_int, vp]
        lib.hcgen_affine.argtypes = [vp, ll, ull, ull, ull, ull, vp]
        lib.hcgen_value_of.argtypes = [vp, vp, ll, vp]
        lib.hcgen_zipf.argtypes = [vp, ll, ull, vp, ll, ull, vp]
        _lib = lib
    return _lib


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"generator launch failed (cudaError {rc})")


def stream_u64(stream: int, seed: int, start: int, n: int):
    import torch
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    _check(load().hcgen_stream(out.data_ptr(), start, n, sm.stream_base(stream, seed), 0, _stream()))
    return out


def stream_u32(stream: int, seed: int, start: int, n: int):
    import torch
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(load().hcgen_stream(out.data_ptr(), start, n, sm.stream_base(stream, seed), 1, _stream()))
    return out


def affine_params(n_pop: int, stream: int, seed: int):
    a = (sm.stream_base(stream, seed) % n_pop) | 1
    while np.gcd(a, n_pop) != 1:
        a += 2
    c = sm.stream_base(stream + 1, seed) % n_pop
    return a, c


def sample_u64(key_stream: int, n_pop: int, n: int, sample_stream: int, seed: int):
    """GPU twin of ``stream_at(key_stream, seed, affine_sample(n_pop, n, sample_stream, seed))``."""
    import torch
    a, c = affine_params(n_pop, sample_stream, seed)
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    _check(load().hcgen_affine(out.data_ptr(), n, n_pop, a, c, sm.stream_base(key_stream, seed), _stream()))
    return out


def value_of(keys):
    import torch
    out = torch.empty_like(keys)
    _check(load().hcgen_value_of(out.data_ptr(), keys.data_ptr(), keys.numel(), _stream()))
    return out


def zipf_keys(table: int, stream: int, n: int, cdf_dev, seed: int = 0):
    """GPU twin of ``recipes.zipf_keys``; ``cdf_dev`` is the float64 CDF as a
    CUDA tensor."""
    import torch
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    salt = (table & 0xFFFF) << 48
    _check(load().hcgen_zipf(out.data_ptr(), n, sm.stream_base(stream, seed), cdf_dev.data_ptr(), cdf_dev.numel(),
                             salt, _stream()))
    return out
