"""Python front end of the hash containers: one ``Table`` per hc_table handle.

Device arrays are torch CUDA tensors passed by ``data_ptr()``; torch only
provides memory and streams.  Keys may be given as any integer tensor whose
element size matches the key type (uint32 keys as int32 or uint32 tensors,
uint64 keys as int64 or uint64 tensors): the bits are what count.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

KEY_BYTES = {L.SET_U32: 4, L.SET_U64: 8, L.MAP_I64_I32: 8, L.MAP_U64_U64: 8}
VAL_BYTES = {L.MAP_I64_I32: 4, L.MAP_U64_U64: 8}
# torch dtypes used for outputs (signed views of the key / value bits)
KEY_TORCH = {4: torch.int32, 8: torch.int64}
KEY_NUMPY = {L.SET_U32: np.uint32, L.SET_U64: np.uint64, L.MAP_I64_I32: np.int64, L.MAP_U64_U64: np.uint64}
VAL_NUMPY = {L.MAP_I64_I32: np.int32, L.MAP_U64_U64: np.uint64}
KIND_NAMES = {"set_u32": L.SET_U32, "set_u64": L.SET_U64, "map_i64_i32": L.MAP_I64_I32, "map_u64_u64": L.MAP_U64_U64}


def _stream_handle(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def to_device(a: np.ndarray, device="cuda") -> torch.Tensor:
    """numpy array -> CUDA tensor with the same bits (unsigned types as signed views)."""
    a = np.ascontiguousarray(a)
    view = {1: np.uint8, 4: np.int32, 8: np.int64}[a.dtype.itemsize] if a.dtype.kind in "ui" else a.dtype
    if a.dtype.itemsize == 1:
        view = np.uint8
    return torch.from_numpy(a.view(view)).to(device)


def to_numpy(t: torch.Tensor, dtype) -> np.ndarray:
    """CUDA/CPU tensor -> numpy array of ``dtype`` with the same bits."""
    return t.detach().cpu().numpy().view(dtype)


def _check_tensor(t: torch.Tensor, nbytes: int, name: str, n: int | None = None):
    """A CUDA tensor, contiguous, with `nbytes`-byte elements and (when `n`
    is given) room for at least n of them: the kernels write outputs by
    index, so a short buffer is refused here."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.element_size() != nbytes or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous with {nbytes}-byte elements")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} elements, {n} needed")


def pack_short3(xyz: torch.Tensor, stream=None) -> torch.Tensor:
    """(n, 3) int16 CUDA tensor of block coordinates -> n packed int64 keys
    (hc_pack_short3) for a map created with HASH_TESCHNER_SHORT3."""
    if not isinstance(xyz, torch.Tensor) or not xyz.is_cuda or xyz.dtype != torch.int16 or not xyz.is_contiguous():
        raise TypeError("xyz must be a contiguous int16 CUDA tensor of shape (n, 3)")
    n = xyz.numel() // 3
    keys = torch.empty(n, dtype=torch.int64, device=xyz.device)
    L.check(L.load().hc_pack_short3(xyz.data_ptr(), n, keys.data_ptr(), _stream_handle(stream)))
    return keys


def unpack_short3(keys: torch.Tensor, stream=None) -> torch.Tensor:
    """Packed int64 keys -> (n, 3) int16 coordinates (hc_unpack_short3)."""
    _check_tensor(keys, 8, "keys")
    xyz = torch.empty((keys.numel(), 3), dtype=torch.int16, device=keys.device)
    L.check(L.load().hc_unpack_short3(keys.data_ptr(), keys.numel(), xyz.data_ptr(), _stream_handle(stream)))
    return xyz


class Table:
    """A fixed-capacity GPU hash set or map (``kind`` in L.SET_U32 .. L.MAP_U64_U64)."""

    def __init__(self, kind, slots: int, bucket_bytes: int = 32, hash_mode: int = L.HASH_MIX64, seed: int = 0,
                 stream=None):
        self.lib = L.load()
        if isinstance(kind, str):
            kind = KIND_NAMES[kind]
        self.kind = kind
        self.key_bytes = KEY_BYTES[kind]
        self.val_bytes = VAL_BYTES.get(kind, 0)
        self.device = torch.device("cuda", torch.cuda.current_device())
        cfg = L.Config(bucket_bytes, hash_mode, seed)
        h = ctypes.c_void_p()
        L.check(self.lib.hc_create(ctypes.byref(h), kind, int(slots), ctypes.byref(cfg), _stream_handle(stream)))
        self.h = h
        self.bucket_bytes = bucket_bytes

    # ---------------------------------------------------------- lifecycle --
    def close(self):
        if getattr(self, "h", None) and self.h.value:
            L.check(self.lib.hc_destroy(self.h))
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def is_map(self) -> bool:
        return self.val_bytes > 0

    @property
    def handle(self) -> int:
        return self.h.value

    def set_launch(self, op: int, lane_bytes: int = 0, keys_per_group: int = 0, block: int = 0, fold: int = 0):
        """fold: 0 keep, 1 on, 2 off."""
        sh = L.Launch(lane_bytes, keys_per_group, block, fold)
        L.check(self.lib.hc_set_launch(self.h, op, ctypes.byref(sh)))

    def get_launch(self, op: int) -> dict:
        sh = L.Launch()
        L.check(self.lib.hc_get_launch(self.h, op, ctypes.byref(sh)))
        return {"lane_bytes": sh.lane_bytes, "keys_per_group": sh.keys_per_group, "block": sh.block,
                "fold": sh.fold_duplicates}

    # ------------------------------------------------------- range calls --
    def insert(self, keys: torch.Tensor, vals: torch.Tensor | None = None, status: torch.Tensor | bool = True,
               stream=None) -> torch.Tensor | None:
        _check_tensor(keys, self.key_bytes, "keys")
        n = keys.numel()
        if self.is_map:
            if vals is None:
                raise TypeError("a map insert needs values")
            _check_tensor(vals, self.val_bytes, "vals")
            if vals.numel() != n:
                raise ValueError("keys and vals differ in length")
        if status is True:
            status = torch.empty(n, dtype=torch.uint8, device=keys.device)
        elif status is False:
            status = None
        if status is not None:
            _check_tensor(status, 1, "status", n)
        L.check(self.lib.hc_insert(self.h, keys.data_ptr(), vals.data_ptr() if self.is_map else None, n,
                                   status.data_ptr() if status is not None else None, _stream_handle(stream)))
        return status

    def insert_if_absent(self, keys: torch.Tensor, vals: torch.Tensor | None, found: torch.Tensor,
                         status: torch.Tensor | bool = True, stream=None) -> torch.Tensor | None:
        """Insert the keys whose ``found`` flag (from ``find`` on the same keys)
        is 0; flagged keys get EXISTS without a probe."""
        _check_tensor(keys, self.key_bytes, "keys")
        n = keys.numel()
        _check_tensor(found, 1, "found", n)
        if self.is_map:
            _check_tensor(vals, self.val_bytes, "vals", n)
        if status is True:
            status = torch.empty(n, dtype=torch.uint8, device=keys.device)
        elif status is False:
            status = None
        if status is not None:
            _check_tensor(status, 1, "status", n)
        L.check(self.lib.hc_insert_if_absent(self.h, keys.data_ptr(), vals.data_ptr() if self.is_map else None,
                                             found.data_ptr(), n, status.data_ptr() if status is not None else None,
                                             _stream_handle(stream)))
        return status

    def apply_mixed(self, ops: torch.Tensor, keys: torch.Tensor, vals: torch.Tensor | None = None,
                    status: torch.Tensor | bool = True, vals_out: torch.Tensor | bool = False, stream=None):
        """Free-running mixed batch (hc_apply_mixed): ops[i] 0 insert, 1 find,
        2 erase, all at once.  Returns (status, vals_out or None)."""
        _check_tensor(ops, 1, "ops")
        _check_tensor(keys, self.key_bytes, "keys")
        n = keys.numel()
        if ops.numel() != n:
            raise ValueError("ops and keys differ in length")
        if self.is_map:
            _check_tensor(vals, self.val_bytes, "vals", n)
        if status is True:
            status = torch.empty(n, dtype=torch.uint8, device=keys.device)
        elif status is False:
            status = None
        if status is not None:
            _check_tensor(status, 1, "status", n)
        if self.is_map and vals_out is True:
            vals_out = torch.empty(n, dtype=KEY_TORCH[self.val_bytes], device=keys.device)
        elif not isinstance(vals_out, torch.Tensor) or not self.is_map:
            vals_out = None
        if vals_out is not None:
            _check_tensor(vals_out, self.val_bytes, "vals_out", n)
        L.check(self.lib.hc_apply_mixed(self.h, ops.data_ptr(), keys.data_ptr(),
                                        vals.data_ptr() if self.is_map else None, n,
                                        status.data_ptr() if status is not None else None,
                                        vals_out.data_ptr() if vals_out is not None else None, _stream_handle(stream)))
        return status, vals_out

    def _scratch(self, n: int, scratch: torch.Tensor | None) -> torch.Tensor:
        need = int(self.lib.hc_ordered_scratch_bytes(n))
        if scratch is None or scratch.numel() < need + 255:     # room to align the base to 256 bytes
            scratch = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        return scratch

    def insert_ordered(self, keys: torch.Tensor, vals: torch.Tensor | None = None, status: torch.Tensor | bool = True,
                       scratch: torch.Tensor | None = None, stream=None) -> torch.Tensor | None:
        """Insert where the lowest index wins among equal keys (every position
        gets the result of a sequential pass in index order)."""
        _check_tensor(keys, self.key_bytes, "keys")
        n = keys.numel()
        if self.is_map:
            _check_tensor(vals, self.val_bytes, "vals", n)
        if status is True:
            status = torch.empty(n, dtype=torch.uint8, device=keys.device)
        elif status is False:
            status = None
        if status is not None:
            _check_tensor(status, 1, "status", n)
        sc = self._scratch(n, scratch)
        base = (sc.data_ptr() + 255) // 256 * 256
        L.check(self.lib.hc_insert_ordered(self.h, keys.data_ptr(), vals.data_ptr() if self.is_map else None, n,
                                           status.data_ptr() if status is not None else None, base,
                                           sc.numel() - (base - sc.data_ptr()), _stream_handle(stream)))
        return status

    def erase_ordered(self, keys: torch.Tensor, status: torch.Tensor | bool = True, scratch: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor | None:
        """Erase where the first occurrence of a key erases it and later ones
        report NOT_FOUND."""
        _check_tensor(keys, self.key_bytes, "keys")
        n = keys.numel()
        if status is True:
            status = torch.empty(n, dtype=torch.uint8, device=keys.device)
        elif status is False:
            status = None
        if status is not None:
            _check_tensor(status, 1, "status", n)
        sc = self._scratch(n, scratch)
        base = (sc.data_ptr() + 255) // 256 * 256
        L.check(self.lib.hc_erase_ordered(self.h, keys.data_ptr(), n, status.data_ptr() if status is not None else None,
                                          base, sc.numel() - (base - sc.data_ptr()), _stream_handle(stream)))
        return status

    def find(self, keys: torch.Tensor, found: torch.Tensor | None = None, vals_out: torch.Tensor | bool | None = True,
             stream=None):
        _check_tensor(keys, self.key_bytes, "keys")
        n = keys.numel()
        if found is None:
            found = torch.empty(n, dtype=torch.uint8, device=keys.device)
        _check_tensor(found, 1, "found", n)
        if self.is_map and vals_out is True:
            vals_out = torch.empty(n, dtype=KEY_TORCH[self.val_bytes], device=keys.device)
        elif vals_out is True or vals_out is False or not self.is_map:
            vals_out = None
        if vals_out is not None:
            _check_tensor(vals_out, self.val_bytes, "vals_out", n)
        L.check(self.lib.hc_find(self.h, keys.data_ptr(), n, found.data_ptr(),
                                 vals_out.data_ptr() if vals_out is not None else None, _stream_handle(stream)))
        return found, vals_out

    def erase(self, keys: torch.Tensor, status: torch.Tensor | bool = True, stream=None) -> torch.Tensor | None:
        _check_tensor(keys, self.key_bytes, "keys")
        n = keys.numel()
        if status is True:
            status = torch.empty(n, dtype=torch.uint8, device=keys.device)
        elif status is False:
            status = None
        if status is not None:
            _check_tensor(status, 1, "status", n)
        L.check(self.lib.hc_erase(self.h, keys.data_ptr(), n, status.data_ptr() if status is not None else None,
                                  _stream_handle(stream)))
        return status

    # ------------------------------------------------- host-buffer calls --
    def _host(self, a: np.ndarray, nbytes: int) -> np.ndarray:
        a = np.ascontiguousarray(a)
        if a.dtype.itemsize != nbytes:
            raise TypeError(f"host array must have {nbytes}-byte elements")
        return a

    @staticmethod
    def _host_out(a: np.ndarray, nbytes: int, n: int, name: str) -> np.ndarray:
        """An output array the library writes in place: C-contiguous,
        writeable, `nbytes`-byte elements, at least n of them."""
        if not isinstance(a, np.ndarray) or not a.flags.c_contiguous or not a.flags.writeable:
            raise TypeError(f"{name} must be a writeable C-contiguous numpy array")
        if a.dtype.itemsize != nbytes:
            raise TypeError(f"{name} must have {nbytes}-byte elements")
        if a.size < n:
            raise ValueError(f"{name} holds {a.size} elements, {n} needed")
        return a

    def insert_host(self, keys: np.ndarray, vals: np.ndarray | None = None, status: np.ndarray | None = None,
                    stream=None) -> np.ndarray:
        keys = self._host(keys, self.key_bytes)
        n = len(keys)
        if self.is_map:
            vals = self._host(vals, self.val_bytes)
            if len(vals) != n:
                raise ValueError("keys and vals differ in length")
        if status is None:
            status = np.empty(n, np.uint8)
        self._host_out(status, 1, n, "status")
        L.check(self.lib.hc_insert_host(self.h, keys.ctypes.data, vals.ctypes.data if self.is_map else None, n,
                                        status.ctypes.data, _stream_handle(stream)))
        return status

    def find_host(self, keys: np.ndarray, found: np.ndarray | None = None, vals_out: np.ndarray | None = None,
                  stream=None):
        keys = self._host(keys, self.key_bytes)
        n = len(keys)
        if found is None:
            found = np.empty(n, np.uint8)
        if self.is_map and vals_out is None:
            vals_out = np.empty(n, VAL_NUMPY[self.kind])
        self._host_out(found, 1, n, "found")
        if self.is_map:
            self._host_out(vals_out, self.val_bytes, n, "vals_out")
        L.check(self.lib.hc_find_host(self.h, keys.ctypes.data, n, found.ctypes.data,
                                      vals_out.ctypes.data if self.is_map else None, _stream_handle(stream)))
        return found, (vals_out if self.is_map else None)

    def erase_host(self, keys: np.ndarray, status: np.ndarray | None = None, stream=None) -> np.ndarray:
        keys = self._host(keys, self.key_bytes)
        n = len(keys)
        if status is None:
            status = np.empty(n, np.uint8)
        self._host_out(status, 1, n, "status")
        L.check(self.lib.hc_erase_host(self.h, keys.ctypes.data, n, status.ctypes.data, _stream_handle(stream)))
        return status

    # ------------------------------------------------------- whole table --
    def select(self, kind: int = L.PRED_ALL, lo: int = 0, hi: int = 0, box=(0, 0, 0, 0, 0, 0), negate: bool = False,
               keys_out: torch.Tensor | None = None, vals_out: torch.Tensor | bool | None = True,
               count: torch.Tensor | None = None, cap: int | None = None, stream=None):
        """Append the stored entries that satisfy the predicate (hc_select) to
        keys_out / vals_out through the device int64 `count` (the output's
        size, 0 when not given).  Returns (keys_out, vals_out, count); no
        synchronisation.  Bounds wrap to int64 as the C struct holds them."""
        if cap is None:
            cap = keys_out.numel() if keys_out is not None else self.size(stream)
        if keys_out is None:
            keys_out = torch.empty(cap, dtype=KEY_TORCH[self.key_bytes], device=self.device)
        if self.is_map and vals_out is True:
            vals_out = torch.empty(cap, dtype=KEY_TORCH[self.val_bytes], device=self.device)
        elif not isinstance(vals_out, torch.Tensor) or not self.is_map:
            vals_out = None
        if count is None:
            count = torch.zeros(1, dtype=torch.int64, device=self.device)
        _check_tensor(count, 8, "count", 1)
        _check_tensor(keys_out, self.key_bytes, "keys_out", cap)
        if vals_out is not None:
            _check_tensor(vals_out, self.val_bytes, "vals_out", cap)
        wrap = lambda x: ((int(x) + 2**63) % 2**64) - 2**63
        pred = L.Predicate(kind, int(negate), wrap(lo), wrap(hi), (ctypes.c_int32 * 6)(*box))
        L.check(self.lib.hc_select(self.h, ctypes.byref(pred), keys_out.data_ptr(),
                                   vals_out.data_ptr() if vals_out is not None else None, cap, count.data_ptr(),
                                   _stream_handle(stream)))
        return keys_out, vals_out, count

    def device_view(self, stream=None) -> L.DeviceView:
        """The hc_device_view that kernels using include/hc_device.cuh take."""
        dv = L.DeviceView()
        L.check(self.lib.hc_device_view_get(self.h, ctypes.byref(dv), _stream_handle(stream)))
        return dv

    def size(self, stream=None) -> int:
        v = ctypes.c_int64()
        L.check(self.lib.hc_size(self.h, ctypes.byref(v), _stream_handle(stream)))
        return v.value

    def stats(self, stream=None) -> dict:
        s = L.Stats()
        L.check(self.lib.hc_stats(self.h, ctypes.byref(s), _stream_handle(stream)))
        return {f: getattr(s, f) for f, _ in L.Stats._fields_ if f != "reserved"}

    def status(self, stream=None) -> int:
        """HC_OK, or the sticky error code (cleared by this call)."""
        rc = self.lib.hc_status(self.h, _stream_handle(stream))
        if rc not in (L.OK, L.ERR_OVERFLOW, L.ERR_STATE):
            L.check(rc)
        return rc

    def clear(self, stream=None):
        L.check(self.lib.hc_clear(self.h, _stream_handle(stream)))

    def rehash(self, new_slots: int, stream=None):
        L.check(self.lib.hc_rehash(self.h, int(new_slots), _stream_handle(stream)))

    def dump(self, stream=None):
        """Stored keys (and values) as device tensors, in unspecified order."""
        n = self.size(stream)
        keys = torch.empty(max(n, 1), dtype=KEY_TORCH[self.key_bytes], device=self.device)
        vals = torch.empty(max(n, 1), dtype=KEY_TORCH[self.val_bytes], device=self.device) if self.is_map else None
        got = ctypes.c_int64()
        L.check(self.lib.hc_dump(self.h, keys.data_ptr(), vals.data_ptr() if vals is not None else None, n,
                                 ctypes.byref(got), _stream_handle(stream)))
        return keys[:got.value], (vals[:got.value] if vals is not None else None)

    def dump_numpy(self, stream=None):
        """Stored (keys, values) as numpy arrays sorted by key bit pattern."""
        k, v = self.dump(stream)
        kn = to_numpy(k, KEY_NUMPY[self.kind])
        order = np.argsort(kn.view(np.uint32 if self.key_bytes == 4 else np.uint64), kind="stable")
        vn = to_numpy(v, VAL_NUMPY[self.kind])[order] if v is not None else None
        return kn[order], vn
