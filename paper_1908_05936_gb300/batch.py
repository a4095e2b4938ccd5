"""Batched form: many range calls on many tables in one persistent launch per
phase (all inserts, then all finds, then all erases), optionally captured once
into a CUDA graph and replayed (hc_batch_* in include/hc.h)."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib as L
from .table import Table, _check_tensor, _stream_handle


@dataclass
class Item:
    """One range call: ``op`` on ``table`` over ``keys`` (and ``vals`` for a
    map insert); results go to ``out`` (status, or found flags for a find) and
    ``vals_out`` (map find values)."""
    table: Table
    op: int
    keys: torch.Tensor
    vals: torch.Tensor | None = None
    out: torch.Tensor | None = None
    vals_out: torch.Tensor | None = None


class Batch:
    def __init__(self, items: list[Item], lane_bytes: int = 0, keys_per_group: int = 0, block: int = 0,
                 blocks_per_sm: int = 0, tile: int = 0, use_graph: bool = True, stream=None):
        self.lib = L.load()
        self.items = list(items)          # keeps every tensor alive while the batch exists
        arr = (L.BatchItem * max(1, len(self.items)))()
        for i, it in enumerate(self.items):
            n = it.keys.numel()
            _check_tensor(it.keys, it.table.key_bytes, "keys")
            if it.vals is not None and it.table.is_map:
                _check_tensor(it.vals, it.table.val_bytes, "vals", n)
            if it.out is not None:
                _check_tensor(it.out, 1, "out", n)
            if it.vals_out is not None and it.table.is_map:
                _check_tensor(it.vals_out, it.table.val_bytes, "vals_out", n)
            arr[i] = L.BatchItem(it.table.handle, it.op, 0, it.keys.data_ptr(),
                                 it.vals.data_ptr() if it.vals is not None else None, it.keys.numel(),
                                 it.out.data_ptr() if it.out is not None else None,
                                 it.vals_out.data_ptr() if it.vals_out is not None else None)
        cfg = L.BatchConfig(lane_bytes, keys_per_group, block, blocks_per_sm, tile, 1 if use_graph else 0)
        h = ctypes.c_void_p()
        L.check(self.lib.hc_batch_create(ctypes.byref(h), arr, len(self.items), ctypes.byref(cfg),
                                         _stream_handle(stream)))
        self.h = h

    def launch(self, stream=None):
        L.check(self.lib.hc_batch_launch(self.h, _stream_handle(stream)))

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            L.check(self.lib.hc_batch_destroy(self.h))
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
