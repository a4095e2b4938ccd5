"""Pins for the CPU oracle: checks against things other than the oracle itself.

* ``SortedArrayModel`` -- brute force on tiny inputs: a sorted Python list
  searched with bisect, capacity counted by scanning it.
* ``stl_results`` -- the C++ standard library's unordered_map /
  unordered_set on the same operation script (library special case; valid
  while the script never reaches the capacity).
* invariants that hold for any correct container: size equals the number of
  distinct stored keys, one INSERTED per distinct new key, erase of all
  inserted keys leaves the container empty, inserting past capacity is
  reported and changes nothing.

``run_all_pins(lib)`` runs every check against an oracle library handle and
returns a list of failure messages; the mutation test uses it to show that a
planted mistake in the oracle is caught.
"""
from __future__ import annotations

import bisect
import os
import random
import shutil
import subprocess
import tempfile

import numpy as np

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))

KINDS = (O.SET_U32, O.SET_U64, O.MAP_I64_I32, O.MAP_U64_U64)
KEY_BITS = {O.SET_U32: 32, O.SET_U64: 64, O.MAP_I64_I32: 64, O.MAP_U64_U64: 64}


def reserved_patterns(kind: int) -> tuple[int, int]:
    """The two largest bit patterns of the key type (all ones, all ones - 1)."""
    top = (1 << KEY_BITS[kind]) - 1
    return top, top - 1


def to_pattern(kind: int, k) -> int:
    return int(k) & ((1 << KEY_BITS[kind]) - 1)


def from_pattern(kind: int, p: int):
    """Bit pattern -> value of the key dtype (int64 keys may be negative)."""
    if kind == O.MAP_I64_I32 and p >= 1 << 63:
        return p - (1 << 64)
    return p


def key_array(kind: int, patterns) -> np.ndarray:
    if kind == O.MAP_I64_I32:
        return np.array([from_pattern(kind, p) for p in patterns], dtype=np.int64)
    return np.array(list(patterns), dtype=O.KEY_DTYPE[kind])


def val_array(kind: int, vals):
    if kind == O.MAP_I64_I32:
        return np.array(vals, dtype=np.int64).astype(np.int32)
    if kind == O.MAP_U64_U64:
        return np.array(vals, dtype=np.uint64)
    return None


class SortedArrayModel:
    """Brute-force container: a sorted list of key bit patterns."""

    def __init__(self, kind: int, capacity: int):
        self.kind, self.cap = kind, capacity
        self.keys: list[int] = []
        self.vals: list[int] = []
        self.res = reserved_patterns(kind)

    def regular_count(self) -> int:
        n = len(self.keys)
        # the reserved patterns are the two largest, so they sort last
        for r in self.res:
            i = bisect.bisect_left(self.keys, r)
            n -= int(i < len(self.keys) and self.keys[i] == r)
        return n

    def insert(self, k: int, v: int) -> int:
        i = bisect.bisect_left(self.keys, k)
        if i < len(self.keys) and self.keys[i] == k:
            return O.EXISTS
        if k not in self.res and self.regular_count() >= self.cap:
            return O.OVERFLOW
        self.keys.insert(i, k)
        self.vals.insert(i, v)
        return O.INSERTED

    def find(self, k: int):
        i = bisect.bisect_left(self.keys, k)
        if i < len(self.keys) and self.keys[i] == k:
            return 1, self.vals[i]
        return 0, 0

    def erase(self, k: int) -> int:
        i = bisect.bisect_left(self.keys, k)
        if i < len(self.keys) and self.keys[i] == k:
            del self.keys[i]
            del self.vals[i]
            return O.ERASED
        return O.NOT_FOUND

    def clear(self):
        self.keys, self.vals = [], []

    def rehash(self, c: int) -> bool:
        if c < 1 or c < self.regular_count():
            return False
        self.cap = c
        return True


def _val_pattern(kind: int, v) -> int:
    if kind == O.MAP_I64_I32:
        return int(np.int64(v)) & 0xFFFFFFFF
    if kind == O.MAP_U64_U64:
        return int(v)
    return 0


def random_script(rng: random.Random, kind: int, n_batches: int, domain: list[int],
                  max_batch: int = 12, with_rehash: bool = True):
    """Batches of (op, key patterns, value patterns)."""
    ops = ["I", "I", "F", "E", "S"] + (["R", "C"] if with_rehash else [])
    script = []
    for _ in range(n_batches):
        op = rng.choice(ops)
        if op in "IFE":
            n = rng.randint(0, max_batch)
            keys = [rng.choice(domain) for _ in range(n)]
            vals = [rng.getrandbits(32 if kind == O.MAP_I64_I32 else 64) for _ in range(n)]
            script.append((op, keys, vals))
        elif op == "R":
            script.append((op, [rng.randint(1, 20)], []))
        else:
            script.append((op, [], []))
    return script


def check_against_brute_force(lib, kind: int, capacity: int, script) -> list[str]:
    """Run a script through the oracle (batched) and the brute force (per key)."""
    errs = []
    t = O.OracleTable(kind, capacity, lib)
    m = SortedArrayModel(kind, capacity)
    for bi, (op, keys, vals) in enumerate(script):
        if op == "I":
            st = t.insert(key_array(kind, keys), val_array(kind, vals) if t.is_map else None)
            exp = [m.insert(k, _val_pattern(kind, v) if t.is_map else 0) for k, v in zip(keys, vals)]
            if list(st) != exp:
                errs.append(f"kind {kind} batch {bi} insert status {list(st)} != {exp}")
        elif op == "F":
            found, fv = t.find(key_array(kind, keys))
            exp = [m.find(k) for k in keys]
            if list(found) != [e[0] for e in exp]:
                errs.append(f"kind {kind} batch {bi} find flags {list(found)} != {[e[0] for e in exp]}")
            if t.is_map:
                got = [_val_pattern(kind, v) for v in fv]
                if got != [e[1] for e in exp]:
                    errs.append(f"kind {kind} batch {bi} find values differ")
        elif op == "E":
            st = t.erase(key_array(kind, keys))
            exp = [m.erase(k) for k in keys]
            if list(st) != exp:
                errs.append(f"kind {kind} batch {bi} erase status {list(st)} != {exp}")
        elif op == "R":
            if t.rehash(keys[0]) != m.rehash(keys[0]):
                errs.append(f"kind {kind} batch {bi} rehash({keys[0]}) acceptance differs")
        elif op == "C":
            t.clear()
            m.clear()
        if t.size() != len(m.keys):
            errs.append(f"kind {kind} batch {bi} size {t.size()} != {len(m.keys)}")
            break
    dk, dv = t.dump()
    got = sorted(zip([to_pattern(kind, k) for k in dk],
                     [_val_pattern(kind, v) for v in dv] if t.is_map else [0] * len(dk)))
    exp = sorted(zip(m.keys, m.vals if t.is_map else [0] * len(m.keys)))
    if got != exp:
        errs.append(f"kind {kind} final contents differ")
    t.close()
    return errs


def tiny_domain(kind: int) -> list[int]:
    top, top1 = reserved_patterns(kind)
    return list(range(16)) + [top, top1, top - 2, 1 << (KEY_BITS[kind] - 1)]


def brute_force_pins(lib, seed: int = 0, n_scripts: int = 40) -> list[str]:
    rng = random.Random(seed)
    errs = []
    for kind in KINDS:
        for s in range(n_scripts):
            cap = rng.randint(1, 16)
            script = random_script(rng, kind, 25, tiny_domain(kind))
            errs += check_against_brute_force(lib, kind, cap, script)
        # wider domain so the oracle's chains hold several nodes
        dom = [rng.getrandbits(KEY_BITS[kind]) for _ in range(3000)] + tiny_domain(kind)
        script = random_script(rng, kind, 300, dom, max_batch=200, with_rehash=False)
        errs += check_against_brute_force(lib, kind, 100000, script)
    return errs


# ----------------------------------------------------------------- STL pin ---

_stl_bin = None


def stl_binary() -> str | None:
    """Compile tests/stl_model.cpp once (None when no C++ compiler exists)."""
    global _stl_bin
    if _stl_bin is None:
        gxx = shutil.which("g++")
        if gxx is None:
            return None
        d = tempfile.mkdtemp(prefix="stl_model_")
        out = os.path.join(d, "stl_model")
        subprocess.run([gxx, "-O2", "-std=c++17", os.path.join(HERE, "stl_model.cpp"), "-o", out], check=True)
        _stl_bin = out
    return _stl_bin


def stl_results(kind: int, script) -> list[str]:
    lines = [str(kind)]
    for op, keys, vals in script:
        if op == "I":
            lines += [f"I {k} {_val_pattern(kind, v) if kind >= 2 else 0}" for k, v in zip(keys, vals)]
        elif op == "F":
            lines += [f"F {k}" for k in keys]
        elif op == "E":
            lines += [f"E {k}" for k in keys]
        elif op == "S":
            lines.append("S")
        elif op == "C":
            lines.append("C")
    out = subprocess.run([stl_binary()], input="\n".join(lines) + "\n", capture_output=True,
                         text=True, check=True).stdout.split("\n")
    return [x for x in out if x]


def oracle_script_results(lib, kind: int, capacity: int, script) -> list[str]:
    t = O.OracleTable(kind, capacity, lib)
    res = []
    for op, keys, vals in script:
        if op == "I":
            st = t.insert(key_array(kind, keys), val_array(kind, vals) if t.is_map else None)
            res += [str(int(s)) for s in st]
        elif op == "F":
            f, v = t.find(key_array(kind, keys))
            for i in range(len(keys)):
                res.append(f"{int(f[i])} {_val_pattern(kind, v[i]) if t.is_map else 0}")
        elif op == "E":
            res += [str(int(s)) for s in t.erase(key_array(kind, keys))]
        elif op == "S":
            res.append(str(t.size()))
        elif op == "C":
            t.clear()
            res.append("ok")
    t.close()
    return res


def stl_pins(lib, seed: int = 1) -> list[str]:
    if stl_binary() is None:
        return []
    rng = random.Random(seed)
    errs = []
    for kind in KINDS:
        dom = tiny_domain(kind) + [rng.getrandbits(KEY_BITS[kind]) for _ in range(200)]
        script = [s for s in random_script(rng, kind, 200, dom, max_batch=40, with_rehash=False)]
        if stl_results(kind, script) != oracle_script_results(lib, kind, 1 << 20, script):
            errs.append(f"kind {kind}: oracle differs from std::unordered_{'map' if kind >= 2 else 'set'}")
    return errs


# ------------------------------------------------------------ invariants ---

def invariant_pins(lib, seed: int = 2) -> list[str]:
    rng = np.random.default_rng(seed)
    errs = []
    for kind in KINDS:
        kdt = O.KEY_DTYPE[kind]
        top, top1 = reserved_patterns(kind)
        # 1. one INSERTED per distinct new key; size = distinct keys
        t = O.OracleTable(kind, 1 << 16, lib)
        keys = rng.integers(0, 500, size=2000).astype(kdt)
        vals = val_array(kind, rng.integers(0, 1 << 31, size=2000)) if t.is_map else None
        st = t.insert(keys, vals)
        ins = keys[st == O.INSERTED]
        if len(ins) != len(np.unique(keys)) or len(np.unique(ins)) != len(ins):
            errs.append(f"kind {kind}: not one INSERTED per distinct key")
        if t.size() != len(np.unique(keys)):
            errs.append(f"kind {kind}: size != distinct keys")
        dk, _ = t.dump()
        if len(dk) != t.size() or len(np.unique(dk)) != len(dk):
            errs.append(f"kind {kind}: dump not a set of size() keys")
        # map value kept from the first insert of each key
        if t.is_map:
            first = {}
            for i, k in enumerate(keys):
                first.setdefault(int(k), _val_pattern(kind, vals[i]))
            f, fv = t.find(np.unique(keys))
            if not f.all() or [_val_pattern(kind, v) for v in fv] != [first[int(k)] for k in np.unique(keys)]:
                errs.append(f"kind {kind}: stored value is not the first inserted one")
        # 2. erase of everything inserted leaves it empty
        es = t.erase(keys)
        if (es == O.ERASED).sum() != len(np.unique(keys)) or t.size() != 0 or len(t.dump()[0]) != 0:
            errs.append(f"kind {kind}: erase-all does not empty the container")
        f, _ = t.find(keys)
        if f.any():
            errs.append(f"kind {kind}: erased key still found")
        t.close()
        # 3. overflow past capacity is reported, changes nothing, spares reserved keys
        cap = 8
        t = O.OracleTable(kind, cap, lib)
        keys = key_array(kind, list(range(100, 100 + cap + 5)) + [top, top1])
        vals = val_array(kind, list(range(len(keys)))) if t.is_map else None
        st = t.insert(keys, vals)
        if list(st) != [O.INSERTED] * cap + [O.OVERFLOW] * 5 + [O.INSERTED] * 2:
            errs.append(f"kind {kind}: overflow statuses wrong {list(st)}")
        f, _ = t.find(keys)
        if list(f) != [1] * cap + [0] * 5 + [1, 1] or t.size() != cap + 2:
            errs.append(f"kind {kind}: overflowed keys stored or size wrong")
        # a present key is EXISTS even when full; erase frees a slot
        if list(t.insert(keys[:1], vals[:1] if vals is not None else None)) != [O.EXISTS]:
            errs.append(f"kind {kind}: present key not EXISTS when full")
        t.erase(keys[:1])
        if list(t.insert(keys[cap:cap + 2], vals[cap:cap + 2] if vals is not None else None)) != [O.INSERTED, O.OVERFLOW]:
            errs.append(f"kind {kind}: freed slot not reusable exactly once")
        # 4. rehash keeps contents, refuses to shrink below the regular keys
        before = t.dump()
        if t.rehash(cap - 1) or not t.rehash(cap + 10):
            errs.append(f"kind {kind}: rehash acceptance wrong")
        after = t.dump()
        if not np.array_equal(before[0], after[0]):
            errs.append(f"kind {kind}: rehash changed contents")
        if list(t.insert(keys[cap + 1:cap + 5], vals[cap + 1:cap + 5] if vals is not None else None)) != [O.INSERTED] * 4:
            errs.append(f"kind {kind}: larger capacity not honoured after rehash")
        t.clear()
        if t.size() != 0 or len(t.dump()[0]) != 0:
            errs.append(f"kind {kind}: clear leaves keys")
        if list(t.insert(keys[:cap], vals[:cap] if vals is not None else None)) != [O.INSERTED] * cap:
            errs.append(f"kind {kind}: clear did not free capacity")
        t.close()
    return errs


def run_all_pins(lib) -> list[str]:
    return brute_force_pins(lib, n_scripts=12) + stl_pins(lib) + invariant_pins(lib)
