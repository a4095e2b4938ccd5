"""Comparison rules between the GPU containers and the CPU oracle.

* contents: the sorted (key, value) lists are equal, bit for bit;
* size: equal;
* find: found flag and value equal at every position;
* insert / erase status: equal as a multiset of (key, status) pairs.  For a
  key that occurs once in the batch this is equality at its position; for a
  key that occurs m > 1 times, which occurrence succeeds is not specified
  under concurrency, so only the multiset of its m statuses is compared
  (exactly one success per distinct key that was absent / present);
* batches that overflow: the invariants of ``check_overflow_insert``.
"""
from __future__ import annotations

import numpy as np

INSERTED, EXISTS, OVERFLOW, ERASED, NOT_FOUND = 0, 1, 2, 3, 4


def bits(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a)
    return a.view({4: np.uint32, 8: np.uint64}[a.dtype.itemsize])


def status_multiset_equal(keys: np.ndarray, got: np.ndarray, exp: np.ndarray) -> bool:
    k = bits(keys).astype(np.uint64)
    g = np.lexsort((got.astype(np.uint64), k))
    e = np.lexsort((exp.astype(np.uint64), k))
    return bool(np.array_equal(k[g], k[e]) and np.array_equal(got[g], exp[e]))


def assert_status(keys, got, exp, what="status"):
    got = np.asarray(got)
    exp = np.asarray(exp)
    assert got.shape == exp.shape, what
    if np.array_equal(got, exp):          # equal at every position: the multisets are equal too
        return
    if not status_multiset_equal(keys, got, exp):
        bad = np.nonzero(got != exp)[0][:10]
        raise AssertionError(f"{what}: (key, status) multisets differ; first differing positions {bad}, "
                             f"got {got[bad]}, expected {exp[bad]}")


def assert_find(got_found, got_vals, exp_found, exp_vals, what="find"):
    got_found = np.asarray(got_found)
    exp_found = np.asarray(exp_found)
    if not np.array_equal(got_found, exp_found):
        bad = np.nonzero(got_found != exp_found)[0][:10]
        raise AssertionError(f"{what}: found flags differ at {bad}")
    if exp_vals is not None:
        if not np.array_equal(bits(got_vals), bits(exp_vals)):
            bad = np.nonzero(bits(got_vals) != bits(exp_vals))[0][:10]
            raise AssertionError(f"{what}: values differ at {bad}")


def assert_contents(got_k, got_v, exp_k, exp_v, what="contents"):
    assert len(got_k) == len(exp_k), f"{what}: {len(got_k)} stored keys, expected {len(exp_k)}"
    assert np.array_equal(bits(got_k), bits(exp_k)), f"{what}: key sets differ"
    if exp_v is not None:
        assert np.array_equal(bits(got_v), bits(exp_v)), f"{what}: values differ"


def check_overflow_insert(keys, status, present_before: set, capacity_free: int, contents_after: set,
                          reserved: set):
    """Invariants of an insert batch that may overflow (the overflowing subset
    is not determined by the semantics):
      - #INSERTED over regular keys = min(#distinct new regular keys, free slots)
      - every reserved (side-slot) new key is INSERTED once
      - every INSERTED key is stored, every OVERFLOW key is absent
      - a key present before is never INSERTED or OVERFLOW
      - at most one INSERTED per distinct key; all statuses in {0, 1, 2}
    """
    kb = [int(x) for x in bits(keys)]
    st = np.asarray(status)
    assert set(np.unique(st)) <= {INSERTED, EXISTS, OVERFLOW}
    new_regular = {k for k in kb if k not in present_before and k not in reserved}
    ins = [k for k, s in zip(kb, st) if s == INSERTED]
    assert len(ins) == len(set(ins)), "a key inserted twice"
    ins_regular = [k for k in ins if k not in reserved]
    assert len(ins_regular) == min(len(new_regular), capacity_free), \
        f"{len(ins_regular)} inserted, expected min({len(new_regular)}, {capacity_free})"
    for k, s in zip(kb, st):
        if s == INSERTED:
            assert k in contents_after and k not in present_before
        elif s == OVERFLOW:
            assert k not in contents_after and k not in reserved
        if k in present_before:
            assert s == EXISTS
    for k in {k for k in kb if k in reserved and k not in present_before}:
        assert k in ins
