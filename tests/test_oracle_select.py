"""Pins of the oracle's selection over stored entries (Section 3.6), on the CPU:
closed forms built from the entries' construction, not from the predicate
code: coordinates enumerated inside a box, residues of a mask, signed versus
unsigned order of the same bit patterns, and the partition of the stored
entries by a predicate and its negation."""
import itertools

import numpy as np

from oracle import oracle as O


def _pack(x, y, z):
    m = (1 << 21) - 1
    return (x & m) | ((y & m) << 21) | ((z & m) << 42)


def _table(kind, keys, vals=None):
    t = O.OracleTable(kind, max(16, 2 * len(keys)))
    t.insert(np.asarray(keys, dtype=O.KEY_DTYPE[kind]),
             None if vals is None else np.asarray(vals, dtype=O.VAL_DTYPE[kind]))
    return t


def test_all_is_the_dump_and_negation_partitions():
    rng = np.random.default_rng(1)
    keys = rng.integers(0, 2**63, size=500, dtype=np.int64)
    vals = rng.integers(-2**31, 2**31, size=500, dtype=np.int64).astype(np.int32)
    t = _table(O.MAP_I64_I32, keys, vals)
    try:
        dk, dv = t.dump()
        k, v = t.select(O.PRED_ALL)
        assert np.array_equal(k, dk) and np.array_equal(v, dv)
        for pk, lo, hi in ((O.PRED_KEY_RANGE, 2**61, 2**62), (O.PRED_VALUE_RANGE, -1000, 2**30),
                           (O.PRED_KEY_MASK, 0b1011, 0b0001)):
            a, _ = t.select(pk, lo, hi)
            b, _ = t.select(pk, lo, hi, negate=True)
            assert len(a) + len(b) == len(dk)
            assert np.array_equal(np.sort(np.concatenate([a, b])), np.sort(dk))
            assert not set(a.tolist()) & set(b.tolist())
    finally:
        t.close()


def test_block_box_equals_enumerated_coordinates():
    coords = list(itertools.product(range(-6, 6), repeat=3))
    keys = [_pack(x, y, z) for x, y, z in coords]
    t = _table(O.MAP_I64_I32, keys, list(range(len(keys))))
    rng = np.random.default_rng(2)
    try:
        for _ in range(20):
            b = []
            for _ in range(3):
                lo, hi = sorted(rng.integers(-8, 8, size=2).tolist())
                b += [lo, hi]
            expected = sorted(_pack(x, y, z) for x in range(b[0], b[1] + 1) for y in range(b[2], b[3] + 1)
                              for z in range(b[4], b[5] + 1) if -6 <= min(x, y, z) and max(x, y, z) < 6)
            k, _ = t.select(O.PRED_BLOCK_BOX, box=b)
            assert sorted(k.tolist()) == expected
    finally:
        t.close()


def test_key_mask_residues_and_signed_order():
    t = _table(O.SET_U64, np.arange(64, dtype=np.uint64))
    try:
        k, _ = t.select(O.PRED_KEY_MASK, 0b111, 0b101)
        assert k.tolist() == [i for i in range(64) if i % 8 == 5]
    finally:
        t.close()
    signed = np.arange(-5, 6, dtype=np.int64)
    m = _table(O.MAP_I64_I32, signed, np.zeros(11, np.int32))
    s = _table(O.SET_U64, signed.view(np.uint64))
    u = _table(O.SET_U32, signed.astype(np.int32).view(np.uint32))
    try:
        assert sorted(m.select(O.PRED_KEY_RANGE, -2, 2)[0].tolist()) == [-2, -1, 0, 1, 2]
        # the same bit patterns as unsigned keys: the negatives are huge
        assert s.select(O.PRED_KEY_RANGE, 0, 2)[0].tolist() == [0, 1, 2]
        assert len(s.select(O.PRED_KEY_RANGE, 2**63, 2**64 - 1)[0]) == 5
        # 32-bit keys: bounds taken mod 2^32
        assert u.select(O.PRED_KEY_RANGE, -3, -1)[0].tolist() == [2**32 - 3, 2**32 - 2, 2**32 - 1]
    finally:
        m.close()
        s.close()
        u.close()


def test_value_range_signed_int32():
    t = _table(O.MAP_I64_I32, np.arange(10, dtype=np.int64), np.arange(-5, 5, dtype=np.int32))
    try:
        k, v = t.select(O.PRED_VALUE_RANGE, -2, 1)
        assert k.tolist() == [3, 4, 5, 6] and v.tolist() == [-2, -1, 0, 1]
    finally:
        t.close()


def test_short3_box_equals_enumerated_coordinates():
    """Packed short3 keys (16-bit fields) built from coordinates near both
    ends of the int16 range: the box selects exactly the enumerated ones."""
    vals = [-32768, -32767, -2, -1, 0, 1, 32766, 32767]
    coords = list(itertools.product(vals, repeat=3))
    keys = [(x & 0xFFFF) | ((y & 0xFFFF) << 16) | ((z & 0xFFFF) << 32) for x, y, z in coords]
    t = _table(O.MAP_I64_I32, keys, list(range(len(keys))))
    try:
        for b in ((-32768, -1, -2, 1, 0, 32767), (-1, 1, -32767, 32766, -32768, -32768)):
            expected = sorted(k for k, (x, y, z) in zip(keys, coords)
                              if b[0] <= x <= b[1] and b[2] <= y <= b[3] and b[4] <= z <= b[5])
            k, _ = t.select(O.PRED_SHORT3_BOX, box=b)
            assert sorted(k.tolist()) == expected and len(expected) > 0
    finally:
        t.close()
