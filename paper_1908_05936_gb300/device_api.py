"""ctypes binding of libhc_examples.so: user kernels that call the in-kernel
function form (include/hc_device.cuh, Section 4.1) on tables created through
the C ABI.  Argument marshalling only; loading fails loudly when the library
has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _lib as L
from .table import Table, _check_tensor, _stream_handle

HERE = os.path.dirname(os.path.abspath(__file__))
EXAMPLES_PATH = os.path.join(HERE, "libhc_examples.so")

_lock = threading.Lock()
_ex = None


def load_examples(path: str = EXAMPLES_PATH) -> ctypes.CDLL:
    global _ex
    with _lock:
        if _ex is None:
            if not os.path.exists(path):
                raise ImportError(f"libhc_examples.so is not built ({path}); run `python -m paper_1908_05936_gb300.build`")
            lib = ctypes.CDLL(path)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            P = ctypes.POINTER
            lib.hcx_apply.restype = i32
            lib.hcx_apply.argtypes = [P(L.DeviceView), vp, i32, vp, vp, i64, vp, vp, vp, i32, vp]
            lib.hcx_update_set.restype = i32
            lib.hcx_update_set.argtypes = [P(L.DeviceView), P(L.DeviceView), vp, i64, vp]
            _ex = lib
    return _ex


def _rc(rc: int, what: str) -> None:
    if rc != L.OK:
        raise L.HCError(rc, what)


def apply(table: Table, keys: torch.Tensor, op: int | torch.Tensor = L.OP_INSERT, vals: torch.Tensor | None = None,
          status: torch.Tensor | None = None, vals_out: torch.Tensor | bool = False, pos_out: torch.Tensor | bool = False,
          block: int = 128, stream=None, view: L.DeviceView | None = None):
    """One in-kernel operation per thread: `op` is 0 insert / 1 find / 2 erase
    for every key, or a uint8 tensor of per-key ops (mixed, free-running).
    Returns (status, vals_out or None, pos_out or None)."""
    ex = load_examples()
    dv = view if view is not None else table.device_view(stream)
    _check_tensor(keys, table.key_bytes, "keys")
    n = keys.numel()
    ops = None
    op_all = 0
    if isinstance(op, torch.Tensor):
        _check_tensor(op, 1, "ops", n)
        ops = op
    else:
        op_all = int(op)
    if status is None:
        status = torch.empty(n, dtype=torch.uint8, device=keys.device)
    _check_tensor(status, 1, "status", n)
    if vals is not None:
        _check_tensor(vals, table.val_bytes, "vals", n)
    if vals_out is True:
        vals_out = torch.empty(n, dtype=torch.int32 if table.val_bytes == 4 else torch.int64, device=keys.device)
    if pos_out is True:
        pos_out = torch.empty(n, dtype=torch.int64, device=keys.device)
    vo = vals_out if isinstance(vals_out, torch.Tensor) else None
    po = pos_out if isinstance(pos_out, torch.Tensor) else None
    if vo is not None:
        _check_tensor(vo, table.val_bytes, "vals_out", n)
    if po is not None:
        _check_tensor(po, 8, "pos_out", n)
    _rc(ex.hcx_apply(ctypes.byref(dv), ops.data_ptr() if ops is not None else None, op_all, keys.data_ptr(),
                     vals.data_ptr() if vals is not None else None, n, status.data_ptr(),
                     vo.data_ptr() if vo is not None else None, po.data_ptr() if po is not None else None, block,
                     _stream_handle(stream)), "hcx_apply")
    return status, vo, po


def update_set(block_map: Table, update: Table, blocks: torch.Tensor, stream=None) -> None:
    """Section 4.1's update-set kernel: each block and its neighbours towards
    -x, -y, -z that `block_map` contains are inserted into `update`."""
    ex = load_examples()
    _check_tensor(blocks, 8, "blocks")
    a, b = block_map.device_view(stream), update.device_view(stream)
    _rc(ex.hcx_update_set(ctypes.byref(a), ctypes.byref(b), blocks.data_ptr(), blocks.numel(), _stream_handle(stream)),
        "hcx_update_set")
