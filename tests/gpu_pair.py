"""A GPU table and a CPU oracle table driven with the same calls."""
from __future__ import annotations

import numpy as np
import torch

import compare as C
from oracle import oracle as O
from paper_1908_05936_gb300.table import Table, to_device, to_numpy

RESERVED = {
    O.SET_U32: (np.uint32(0xFFFFFFFF), np.uint32(0xFFFFFFFE)),
    O.SET_U64: (np.uint64(2**64 - 1), np.uint64(2**64 - 2)),
    O.MAP_I64_I32: (np.int64(-1), np.int64(-2)),
    O.MAP_U64_U64: (np.uint64(2**64 - 1), np.uint64(2**64 - 2)),
}

# The pattern an in-kernel map insert writes into the slot it claims, before
# the value and the key (all ones minus two).  It is an ordinary key: held in
# a slot, counted against the capacity, and found where the table header
# records it; the test domains carry it so that every path meets it.
CLAIM_PATTERN = {
    O.SET_U32: np.uint32(0xFFFFFFFD),
    O.SET_U64: np.uint64(2**64 - 3),
    O.MAP_I64_I32: np.int64(-3),
    O.MAP_U64_U64: np.uint64(2**64 - 3),
}


def edge_keys(kind: int) -> np.ndarray:
    """The two side-slot patterns and the claim pattern of `kind`."""
    return np.array(list(RESERVED[kind]) + [CLAIM_PATTERN[kind]], dtype=O.KEY_DTYPE[kind])


def random_keys(kind: int, n: int, rng: np.random.Generator, domain: np.ndarray | None = None) -> np.ndarray:
    kdt = O.KEY_DTYPE[kind]
    if domain is not None:
        return domain[rng.integers(0, len(domain), size=n)]
    bits = 32 if kind == O.SET_U32 else 64
    raw = rng.integers(0, 2**bits, size=n, dtype=np.uint64 if bits == 64 else np.uint32)
    return raw.view(kdt) if raw.dtype.itemsize == np.dtype(kdt).itemsize else raw.astype(kdt)


def value_for(kind: int, keys: np.ndarray, salt: int = 0) -> np.ndarray | None:
    """Map values as a fixed function of (key, salt): equal keys inside one
    batch carry equal values, so the stored value does not depend on which
    duplicate wins; a different salt per batch still exercises the rule that
    inserting a present key keeps its old value."""
    if kind not in O.VAL_DTYPE:
        return None
    from workloads import splitmix
    k = np.ascontiguousarray(keys)
    k64 = k.view(np.uint32).astype(np.uint64) if k.dtype.itemsize == 4 else k.view(np.uint64)
    v = splitmix.value_of(k64 ^ np.uint64(salt))
    if kind == O.MAP_I64_I32:
        return (v & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)
    return v


class Pair:
    def __init__(self, kind: int, slots: int, bucket_bytes: int = 32, hash_mode: int = 0, seed: int = 0,
                 shape: dict | None = None):
        self.kind = kind
        self.g = Table(kind, slots, bucket_bytes=bucket_bytes, hash_mode=hash_mode, seed=seed)
        self.o = O.OracleTable(kind, slots)
        if shape:
            shape = dict(shape)
            krb = self.g.get_launch(0)["lane_bytes"]          # default lane = whole key region
            lb = shape.get("lane_bytes", 0)
            if lb == "full":                                   # maps: keys and values in one read
                lb = bucket_bytes if kind in O.VAL_DTYPE else krb
            elif lb == "wide":
                lb = krb
            elif lb == "mid":
                lb = max(krb // 2, 16 if kind in O.VAL_DTYPE else 32)
            elif lb == "narrow":
                lb = 16 if kind in O.VAL_DTYPE else 32
            else:
                lb = min(int(lb), krb)
            shape["lane_bytes"] = lb
            for op in (0, 1, 2):
                self.g.set_launch(op, **shape)
        self.is_map = self.g.is_map

    def close(self):
        self.g.close()
        self.o.close()

    def insert(self, keys, vals=None, check=True):
        gs = self.g.insert(to_device(keys), to_device(vals) if self.is_map else None)
        os_ = self.o.insert(keys, vals)
        gs = to_numpy(gs, np.uint8)
        if check:
            C.assert_status(keys, gs, os_, "insert status")
        return gs, os_

    def find(self, keys):
        gf, gv = self.g.find(to_device(keys))
        of, ov = self.o.find(keys)
        gf = to_numpy(gf, np.uint8)
        gv = to_numpy(gv, O.VAL_DTYPE[self.kind]) if self.is_map else None
        C.assert_find(gf, gv, of, ov)
        return gf, gv

    def erase(self, keys, check=True):
        gs = to_numpy(self.g.erase(to_device(keys)), np.uint8)
        os_ = self.o.erase(keys)
        if check:
            C.assert_status(keys, gs, os_, "erase status")
        return gs, os_

    def clear(self):
        self.g.clear()
        self.o.clear()

    def rehash(self, s: int) -> bool:
        ok_o = self.o.rehash(s)
        try:
            self.g.rehash(s)
            ok_g = True
        except Exception:
            ok_g = False
        assert ok_g == ok_o, f"rehash({s}) accepted by gpu={ok_g} oracle={ok_o}"
        return ok_o

    def check(self):
        assert self.g.size() == self.o.size(), (self.g.size(), self.o.size())
        assert not self.g.stats()["error_bits"] & 4, "a bounds check of the debug build failed"
        gk, gv = self.g.dump_numpy()
        ok, ov = self.o.dump()
        C.assert_contents(gk, gv, ok, ov)
        torch.cuda.synchronize()
