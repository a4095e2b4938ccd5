"""The per-key serial-order rule used by the free-running in-kernel tests,
pinned against a brute force over every order of the operations."""
import random

import numpy as np

import linearizable as LZ


def _random_result(op, rng, overflow=False):
    if op == LZ.OP_INSERT:
        return rng.choice([LZ.INSERTED, LZ.EXISTS, LZ.OVERFLOW] if overflow else [LZ.INSERTED, LZ.EXISTS])
    if op == LZ.OP_ERASE:
        return rng.choice([LZ.ERASED, LZ.NOT_FOUND])
    return rng.choice([0, 1])


def test_counting_rule_equals_brute_force():
    rng = random.Random(7)
    agree = {True: 0, False: 0}
    for _ in range(4000):
        n = rng.randint(0, 6)
        ops = []
        for _ in range(n):
            o = rng.choice([LZ.OP_INSERT, LZ.OP_FIND, LZ.OP_ERASE])
            ops.append((o, _random_result(o, rng)))
        before, after = rng.randint(0, 1), rng.randint(0, 1)
        want = LZ.serial_order_exists(before, after, ops)
        assert LZ.key_ok(before, after, ops) == want, (before, after, ops)
        agree[want] += 1
    assert agree[True] > 200 and agree[False] > 200     # both outcomes exercised


def test_counting_rule_with_overflow_equals_brute_force():
    """Histories of a table that fills up: an insert may report OVERFLOW
    (observed the key absent, changed nothing)."""
    rng = random.Random(9)
    agree = {True: 0, False: 0}
    for _ in range(4000):
        ops = []
        for _ in range(rng.randint(0, 6)):
            o = rng.choice([LZ.OP_INSERT, LZ.OP_FIND, LZ.OP_ERASE])
            ops.append((o, _random_result(o, rng, overflow=True)))
        before, after = rng.randint(0, 1), rng.randint(0, 1)
        want = LZ.serial_order_exists(before, after, ops, overflow=True)
        assert LZ.key_ok(before, after, ops, overflow=True) == want, (before, after, ops)
        agree[want] += 1
    assert agree[True] > 200 and agree[False] > 200
    I = LZ.OP_INSERT
    assert LZ.key_ok(0, 0, [(I, LZ.OVERFLOW)], overflow=True)
    assert not LZ.key_ok(1, 1, [(I, LZ.OVERFLOW)], overflow=True)      # present: EXISTS, not OVERFLOW
    assert LZ.key_ok(0, 1, [(I, LZ.OVERFLOW), (I, LZ.INSERTED)], overflow=True)


def test_serial_runs_pass_and_single_flips_are_judged_like_brute_force():
    rng = random.Random(11)
    for _ in range(1000):
        before = rng.randint(0, 1)
        state, ops = before, []
        for _ in range(rng.randint(1, 6)):
            o = rng.choice([LZ.OP_INSERT, LZ.OP_FIND, LZ.OP_ERASE])
            if o == LZ.OP_INSERT:
                ops.append((o, LZ.EXISTS if state else LZ.INSERTED))
                state = 1
            elif o == LZ.OP_ERASE:
                ops.append((o, LZ.ERASED if state else LZ.NOT_FOUND))
                state = 0
            else:
                ops.append((o, state))
        rng.shuffle(ops)
        assert LZ.key_ok(before, state, ops)
        i = rng.randrange(len(ops))
        o, r = ops[i]
        flipped = {LZ.INSERTED: LZ.EXISTS, LZ.EXISTS: LZ.INSERTED, LZ.ERASED: LZ.NOT_FOUND,
                   LZ.NOT_FOUND: LZ.ERASED, 0: 1, 1: 0}[r] if o != LZ.OP_FIND else 1 - r
        bad = ops[:i] + [(o, flipped)] + ops[i + 1:]
        assert LZ.key_ok(before, state, bad) == LZ.serial_order_exists(before, state, bad)


def test_hand_cases():
    I, F, E = LZ.OP_INSERT, LZ.OP_FIND, LZ.OP_ERASE
    # two inserts of an absent key: exactly one may succeed
    assert LZ.key_ok(0, 1, [(I, LZ.INSERTED), (I, LZ.EXISTS)])
    assert not LZ.key_ok(0, 1, [(I, LZ.INSERTED), (I, LZ.INSERTED)])
    # insert and erase racing on an absent key, key gone afterwards
    assert LZ.key_ok(0, 0, [(I, LZ.INSERTED), (E, LZ.ERASED)])
    assert LZ.key_ok(0, 1, [(I, LZ.INSERTED), (E, LZ.NOT_FOUND)])
    assert not LZ.key_ok(0, 0, [(I, LZ.INSERTED), (E, LZ.NOT_FOUND)])
    # a find that saw the key present needs a present state
    assert not LZ.key_ok(0, 0, [(F, 1), (E, LZ.NOT_FOUND)])
    assert LZ.key_ok(1, 0, [(F, 1), (E, LZ.ERASED), (F, 0)])
    # OVERFLOW is never a valid result in these histories
    assert not LZ.key_ok(0, 0, [(I, LZ.OVERFLOW)])


def test_check_history_groups_keys():
    keys = np.array([5, 9, 5, 9, 9], dtype=np.uint64)
    ops = np.array([0, 0, 0, 2, 1], dtype=np.uint8)
    res = np.array([LZ.INSERTED, LZ.EXISTS, LZ.EXISTS, LZ.ERASED, 0], dtype=np.uint8)
    assert LZ.check_history(keys, ops, res, before={9}, after={5}) == []
    assert LZ.check_history(keys, ops, res, before=set(), after={5}) == [9]
