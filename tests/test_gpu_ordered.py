"""Ordered insert / erase (the lowest index wins among equal keys): every
position equals the sequential oracle exactly, not only as a multiset, and a
map keeps the first occurrence's value even when equal keys carry different
values; overflow keeps the invariants and later occurrences mirror the
first one."""
import numpy as np
import pytest
import torch

import compare as C
from gpu_pair import RESERVED, Pair, edge_keys, random_keys
from oracle import oracle as O
from paper_1908_05936_gb300 import _lib as L
from paper_1908_05936_gb300.table import Table, to_device, to_numpy

pytestmark = pytest.mark.gpu

KINDS = (O.SET_U32, O.SET_U64, O.MAP_I64_I32, O.MAP_U64_U64)


def _values(kind, n, rng):
    """One value per position (equal keys get different values)."""
    if kind == O.MAP_I64_I32:
        return rng.integers(-2**31, 2**31, size=n, dtype=np.int64).astype(np.int32)
    if kind == O.MAP_U64_U64:
        return rng.integers(0, 2**63, size=n, dtype=np.int64).view(np.uint64)
    return None


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bb", (32, 128))
def test_ordered_equals_sequential(kind, bb):
    rng = np.random.default_rng(1100 + kind * 3 + bb)
    p = Pair(kind, 40000, bucket_bytes=bb)
    dom = np.concatenate([random_keys(kind, 3000, rng), edge_keys(kind)])
    try:
        for n in (0, 1, 2, 255, 256, 257, 10000, 20000):
            keys = dom[rng.integers(0, len(dom), size=n)]
            vals = _values(kind, n, rng)
            gs = to_numpy(p.g.insert_ordered(to_device(keys), to_device(vals) if vals is not None else None),
                          np.uint8)
            os_ = p.o.insert(keys, vals)
            assert np.array_equal(gs, os_), "ordered insert differs from the sequential pass"
            er = dom[rng.integers(0, len(dom), size=n // 2)]
            ge = to_numpy(p.g.erase_ordered(to_device(er)), np.uint8)
            assert np.array_equal(ge, p.o.erase(er)), "ordered erase differs from the sequential pass"
            p.check()
        # a lock-step insert shape takes the same skip flags
        p.g.set_launch(L.OP_INSERT, keys_per_group=1)
        keys = dom[rng.integers(0, len(dom), size=5000)]
        vals = _values(kind, 5000, rng)
        gs = to_numpy(p.g.insert_ordered(to_device(keys), to_device(vals) if vals is not None else None), np.uint8)
        assert np.array_equal(gs, p.o.insert(keys, vals))
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("kind", (O.SET_U64, O.MAP_U64_U64))
def test_ordered_overflow_mirrors_first_occurrence(kind):
    rng = np.random.default_rng(1200 + kind)
    t = Table(kind, 100, bucket_bytes=32)
    try:
        keys = random_keys(kind, 300, rng)
        keys = np.concatenate([keys, keys[rng.integers(0, 300, size=300)]])   # every key up to several times
        rng.shuffle(keys)
        vals = _values(kind, len(keys), rng)
        st = to_numpy(t.insert_ordered(to_device(keys), to_device(vals) if vals is not None else None), np.uint8)
        gk, _ = t.dump_numpy()
        C.check_overflow_insert(keys, st, set(), 100, {int(x) for x in C.bits(gk)}, set())
        first = {}
        for k, s in zip(C.bits(keys).tolist(), st.tolist()):
            if k not in first:
                first[k] = s
                assert s in (C.INSERTED, C.OVERFLOW)
            else:
                assert s == (C.OVERFLOW if first[k] == C.OVERFLOW else C.EXISTS)
    finally:
        t.close()


def test_ordered_scratch_checks():
    t = Table(O.SET_U64, 1000)
    try:
        keys = to_device(np.arange(10, dtype=np.uint64))
        lib = t.lib
        need = lib.hc_ordered_scratch_bytes(10)
        assert need >= 10 * 17 and need % 256 == 0
        sc = torch.empty(need, dtype=torch.uint8, device="cuda")
        assert lib.hc_insert_ordered(t.h, keys.data_ptr(), None, 10, None, sc.data_ptr(), need - 256, None) == L.ERR_ARG
        assert lib.hc_insert_ordered(t.h, keys.data_ptr(), None, 10, None, None, need, None) == L.ERR_ARG
        assert lib.hc_insert_ordered(t.h, keys.data_ptr(), None, 10, None, sc.data_ptr(), need, None) == L.OK
        torch.cuda.synchronize()
        assert t.size() == 10
    finally:
        t.close()
