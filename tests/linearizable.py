"""Per-key check of concurrent set operations (host logic for the free-running
tests of the in-kernel API).

The paper's guarantee (Section 4, "Guarantees") is that every operation may
run concurrently with every other.  Keys are independent, so a history of one
concurrent launch is correct when, for every key, its operations' results are
those of SOME serial order of them, starting from the key's presence before the
launch and ending in its presence after it.  All operations of one launch
overlap in time, so any order is allowed.

For a key, let a = inserts that reported INSERTED and e = erases that reported
ERASED.  A serial order exists exactly when
  * the successful inserts and erases alternate from the initial state:
    a - e == after - before (each 0 or 1);
  * operations that observed the key present (insert EXISTS, find found) have
    a present state to sit in: before == 1 or a >= 1;
  * operations that observed it absent (erase NOT_FOUND, find not found) have
    an absent state: before == 0 or e >= 1.
`serial_order_exists` decides the same question by trying every order; the
tests pin the counting rule against it.

With `overflow=True` (a launch on a table that fills up) an insert may also
report OVERFLOW: it found neither the key nor a free slot, so it observed the
key absent and changed nothing.
"""
from __future__ import annotations

import itertools

import numpy as np

INSERTED, EXISTS, OVERFLOW, ERASED, NOT_FOUND = 0, 1, 2, 3, 4
OP_INSERT, OP_FIND, OP_ERASE = 0, 1, 2


def key_ok(before: int, after: int, ops: list[tuple[int, int]], overflow: bool = False) -> bool:
    """Counting rule for one key: ops are (op, result) with find results 1/0."""
    a = sum(1 for o, r in ops if o == OP_INSERT and r == INSERTED)
    e = sum(1 for o, r in ops if o == OP_ERASE and r == ERASED)
    ins_ok = (INSERTED, EXISTS, OVERFLOW) if overflow else (INSERTED, EXISTS)
    if any(o == OP_INSERT and r not in ins_ok for o, r in ops):
        return False
    if any(o == OP_ERASE and r not in (ERASED, NOT_FOUND) for o, r in ops):
        return False
    if a - e != after - before:
        return False
    saw_present = any((o == OP_INSERT and r == EXISTS) or (o == OP_FIND and r == 1) for o, r in ops)
    saw_absent = any((o == OP_ERASE and r == NOT_FOUND) or (o == OP_FIND and r == 0) or
                     (o == OP_INSERT and r == OVERFLOW) for o, r in ops)
    if saw_present and not (before == 1 or a >= 1):
        return False
    if saw_absent and not (before == 0 or e >= 1):
        return False
    return True


def serial_order_exists(before: int, after: int, ops: list[tuple[int, int]], overflow: bool = False) -> bool:
    """Brute force: some permutation of ops, run on a one-key set, gives
    every recorded result and ends in `after`.  With `overflow`, an insert
    of the absent key may fail with OVERFLOW (a full table) instead."""
    for perm in itertools.permutations(ops):
        state, good = before, True
        for o, r in perm:
            if o == OP_INSERT:
                if overflow and r == OVERFLOW and not state:
                    continue                            # absent, table full: nothing changes
                want = EXISTS if state else INSERTED
                state = 1
            elif o == OP_ERASE:
                want = ERASED if state else NOT_FOUND
                state = 0
            else:
                want = state
            if r != want:
                good = False
                break
        if good and state == after:
            return True
    return False


def check_history(keys: np.ndarray, ops: np.ndarray, results: np.ndarray, before: set, after: set,
                  overflow: bool = False) -> list:
    """Keys whose operations in one concurrent launch admit no serial order.
    keys/ops/results are per-thread arrays; before/after are the stored key
    sets (as Python ints) around the launch; `overflow` admits inserts that
    found the table full."""
    bad = []
    order = np.argsort(keys, kind="stable")
    ks, os_, rs = keys[order], ops[order], results[order]
    starts = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]])
    ends = np.r_[starts[1:], len(ks)]
    for s, t in zip(starts, ends):
        k = int(ks[s])
        hist = list(zip(os_[s:t].tolist(), rs[s:t].tolist()))
        if not key_ok(int(k in before), int(k in after), hist, overflow):
            bad.append(k)
    return bad
