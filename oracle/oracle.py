"""ctypes front end of the CPU oracle (hc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  See hc_oracle.c for what
the oracle computes and which passages of the paper it follows.

``OracleTable`` mirrors the container calls: insert / find / erase / size /
clear / rehash / dump, each over a whole numpy batch processed sequentially in
index order.  ``mixed`` applies a batch holding several kinds of operation as
three phases -- every insert, then every find, then every erase -- which is
the order the batched GPU launch defines for one table.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hc_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

SET_U32, SET_U64, MAP_I64_I32, MAP_U64_U64 = 0, 1, 2, 3
INSERTED, EXISTS, OVERFLOW, ERASED, NOT_FOUND = 0, 1, 2, 3, 4

PRED_ALL, PRED_KEY_RANGE, PRED_VALUE_RANGE, PRED_KEY_MASK, PRED_BLOCK_BOX, PRED_SHORT3_BOX = 0, 1, 2, 3, 4, 5

KEY_DTYPE = {SET_U32: np.uint32, SET_U64: np.uint64, MAP_I64_I32: np.int64, MAP_U64_U64: np.uint64}
VAL_DTYPE = {MAP_I64_I32: np.int32, MAP_U64_U64: np.uint64}

_lock = threading.Lock()
_lib = None


def build(src: str = SRC, out: str = LIB, extra_flags: tuple = ()) -> str:
    """Compile the oracle with gcc (-O2, no architecture-specific flags)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", *extra_flags, src, "-o", out]
    subprocess.run(cmd, check=True)
    return out


def _stale() -> bool:
    return not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC)


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (building if needed) the oracle shared library."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            if _stale():
                build()
            _lib = _declare(ctypes.CDLL(LIB))
    return _lib


def _declare(lib: ctypes.CDLL) -> ctypes.CDLL:
    vp, i64, u8p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
    lib.o_create.restype = vp
    lib.o_create.argtypes = [ctypes.c_int, i64]
    lib.o_destroy.argtypes = [vp]
    lib.o_insert.argtypes = [vp, vp, vp, i64, u8p]
    lib.o_find.argtypes = [vp, vp, i64, u8p, vp]
    lib.o_erase.argtypes = [vp, vp, i64, u8p]
    for f in (lib.o_size, lib.o_size_regular, lib.o_capacity):
        f.restype = i64
        f.argtypes = [vp]
    lib.o_clear.argtypes = [vp]
    lib.o_rehash.restype = ctypes.c_int
    lib.o_rehash.argtypes = [vp, i64]
    lib.o_dump.restype = i64
    lib.o_dump.argtypes = [vp, vp, vp, i64]
    return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleTable:
    """Sequential reference container of one kind and capacity."""

    def __init__(self, kind: int, capacity: int, lib: ctypes.CDLL | None = None):
        self.kind = kind
        self.lib = lib if lib is not None else load()
        self.h = self.lib.o_create(kind, capacity)
        if not self.h:
            raise ValueError(f"bad oracle table arguments kind={kind} capacity={capacity}")
        self.kdt = KEY_DTYPE[kind]
        self.vdt = VAL_DTYPE.get(kind)

    @property
    def is_map(self) -> bool:
        return self.vdt is not None

    def close(self):
        if self.h:
            self.lib.o_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _keys(self, keys) -> np.ndarray:
        return np.ascontiguousarray(np.asarray(keys, dtype=self.kdt))

    def insert(self, keys, vals=None) -> np.ndarray:
        k = self._keys(keys)
        v = None
        if self.is_map:
            v = np.ascontiguousarray(np.asarray(vals, dtype=self.vdt))
            assert v.shape == k.shape
        st = np.empty(len(k), np.uint8)
        self.lib.o_insert(self.h, _ptr(k), _ptr(v), len(k), _ptr(st))
        return st

    def find(self, keys):
        k = self._keys(keys)
        found = np.empty(len(k), np.uint8)
        vals = np.empty(len(k), self.vdt) if self.is_map else None
        self.lib.o_find(self.h, _ptr(k), len(k), _ptr(found), _ptr(vals))
        return found, vals

    def erase(self, keys) -> np.ndarray:
        k = self._keys(keys)
        st = np.empty(len(k), np.uint8)
        self.lib.o_erase(self.h, _ptr(k), len(k), _ptr(st))
        return st

    def mixed(self, ins_keys, ins_vals, find_keys, erase_keys):
        """Phase semantics of one batch holding several kinds of operation."""
        a = self.insert(ins_keys, ins_vals)
        b = self.find(find_keys)
        c = self.erase(erase_keys)
        return a, b, c

    def size(self) -> int:
        return int(self.lib.o_size(self.h))

    def size_regular(self) -> int:
        return int(self.lib.o_size_regular(self.h))

    def capacity(self) -> int:
        return int(self.lib.o_capacity(self.h))

    def clear(self):
        self.lib.o_clear(self.h)

    def rehash(self, new_capacity: int) -> bool:
        return self.lib.o_rehash(self.h, new_capacity) == 0

    def dump(self):
        """Stored (keys, values) sorted by key bit pattern (values None for sets)."""
        n = int(self.lib.o_dump(self.h, None, None, 0))
        k = np.empty(n, self.kdt)
        v = np.empty(n, self.vdt) if self.is_map else None
        self.lib.o_dump(self.h, _ptr(k), _ptr(v), n)
        order = np.argsort(k.view(np.uint32 if self.kdt == np.uint32 else np.uint64), kind="stable")
        return k[order], (v[order] if v is not None else None)

    def select(self, pred_kind: int, lo: int = 0, hi: int = 0, box=(0, 0, 0, 0, 0, 0), negate: bool = False):
        """Stored (keys, values) that satisfy the predicate (Section 3.6: a
        range over the stored entries copied with a predicate), sorted by key
        bit pattern."""
        k, v = self.dump()
        keep = [selected(self.kind, pred_kind, lo, hi, box, negate, int(k[i]), None if v is None else int(v[i]))
                for i in range(len(k))]
        keep = np.array(keep, dtype=bool)
        return k[keep], (v[keep] if v is not None else None)


def _block_coord(key_bits: int, field: int) -> int:
    """Signed 21-bit field `field` (0 = x, 1 = y, 2 = z) of a packed block key."""
    c = (key_bits >> (21 * field)) & 0x1FFFFF
    return c - (1 << 21) if c >= (1 << 20) else c


def _short_coord(key_bits: int, field: int) -> int:
    """Signed 16-bit field `field` of a packed short3 key (Section 4.1's
    block coordinates as (uint16)x | (uint16)y << 16 | (uint16)z << 32)."""
    c = (key_bits >> (16 * field)) & 0xFFFF
    return c - (1 << 16) if c >= (1 << 15) else c


def selected(kind: int, pred_kind: int, lo: int, hi: int, box, negate: bool, key: int, val) -> bool:
    """One entry against one predicate.  `key` and `val` are the entry's
    values in the container's own types (int64 keys and int32 values signed,
    the others unsigned); bounds are compared in those types."""
    kbits = key & 0xFFFFFFFFFFFFFFFF
    if pred_kind == PRED_ALL:
        r = True
    elif pred_kind == PRED_KEY_RANGE:
        if kind == MAP_I64_I32:
            r = lo <= key <= hi
        elif kind == SET_U32:
            r = (lo & 0xFFFFFFFF) <= key <= (hi & 0xFFFFFFFF)
        else:
            r = (lo & 0xFFFFFFFFFFFFFFFF) <= key <= (hi & 0xFFFFFFFFFFFFFFFF)
    elif pred_kind == PRED_VALUE_RANGE:
        if kind == MAP_I64_I32:
            r = lo <= val <= hi
        else:
            r = (lo & 0xFFFFFFFFFFFFFFFF) <= val <= (hi & 0xFFFFFFFFFFFFFFFF)
    elif pred_kind == PRED_KEY_MASK:
        r = (kbits & (lo & 0xFFFFFFFFFFFFFFFF)) == (hi & 0xFFFFFFFFFFFFFFFF)
    elif pred_kind == PRED_BLOCK_BOX:
        x, y, z = (_block_coord(kbits, f) for f in range(3))
        r = box[0] <= x <= box[1] and box[2] <= y <= box[3] and box[4] <= z <= box[5]
    elif pred_kind == PRED_SHORT3_BOX:
        x, y, z = (_short_coord(kbits, f) for f in range(3))
        r = box[0] <= x <= box[1] and box[2] <= y <= box[3] and box[4] <= z <= box[5]
    else:
        raise ValueError(f"unknown predicate kind {pred_kind}")
    return r != bool(negate)
