"""hc_select (Section 3.6: stored entries copied with a predicate through a
back inserter) against the oracle's selection, for every kind, bucket size
and predicate, with side-slot keys, tombstones and negation; appending
through the device count, and entries past the output's capacity counted
but not written."""
import itertools

import numpy as np
import pytest
import torch

import compare as C
from gpu_pair import RESERVED, Pair, random_keys, value_for
from oracle import oracle as O
from paper_1908_05936_gb300 import _lib as L
from paper_1908_05936_gb300.table import to_numpy

pytestmark = pytest.mark.gpu

KINDS = (O.SET_U32, O.SET_U64, O.MAP_I64_I32, O.MAP_U64_U64)


def _pack(c):
    m = (1 << 21) - 1
    return (c[:, 0] & m) | ((c[:, 1] & m) << 21) | ((c[:, 2] & m) << 42)


def _gpu_select(p, **kw):
    ko, vo, cnt = p.g.select(**kw)
    n = int(cnt.item())
    gk = to_numpy(ko[:n], O.KEY_DTYPE[p.kind])
    gv = to_numpy(vo[:n], O.VAL_DTYPE[p.kind]) if p.is_map else None
    return gk, gv, n


def _assert_same(p, gk, gv, ok, ov):
    order = np.argsort(C.bits(gk), kind="stable")
    C.assert_contents(gk[order], gv[order] if gv is not None else None, ok, ov, "selection")


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bb", (32, 64, 128))
def test_select_matches_oracle(kind, bb):
    rng = np.random.default_rng(900 + kind * 5 + bb)
    p = Pair(kind, 30000, bucket_bytes=bb)
    try:
        keys = random_keys(kind, 12000, rng)
        if kind != O.SET_U32:
            grid = np.array(list(itertools.product(range(-4, 4), repeat=3)), dtype=np.int64)
            keys = np.concatenate([keys, _pack(grid).astype(np.int64).view(O.KEY_DTYPE[kind])])
        keys = np.concatenate([keys, np.array(RESERVED[kind])])
        p.insert(keys, value_for(kind, keys))
        p.erase(keys[::4])
        srt = np.sort(C.bits(keys))
        preds = [dict(kind=L.PRED_ALL), dict(kind=L.PRED_KEY_MASK, lo=0b1011, hi=0b0010),
                 dict(kind=L.PRED_KEY_MASK, lo=0b1011, hi=0b0010, negate=True)]
        for _ in range(3):
            a, b = sorted(int(x) for x in srt[rng.integers(0, len(srt), size=2)])
            if kind == O.MAP_I64_I32:      # the range is taken in the signed key type
                a, b = sorted(((a + 2**63) % 2**64) - 2**63 for a in (a, b))
            preds += [dict(kind=L.PRED_KEY_RANGE, lo=a, hi=b), dict(kind=L.PRED_KEY_RANGE, lo=a, hi=b, negate=True)]
        if p.is_map:
            if kind == O.MAP_I64_I32:
                preds += [dict(kind=L.PRED_VALUE_RANGE, lo=-2**30, hi=2**29)]
            else:
                preds += [dict(kind=L.PRED_VALUE_RANGE, lo=2**62, hi=2**63 + 2**61)]
        if kind != O.SET_U32:
            preds += [dict(kind=L.PRED_BLOCK_BOX, box=(-2, 1, -4, 3, 0, 0)),
                      dict(kind=L.PRED_BLOCK_BOX, box=(-3, -1, -1, 2, -4, 3), negate=True)]
        for pr in preds:
            gk, gv, n = _gpu_select(p, **pr)
            ok, ov = p.o.select(pr["kind"], pr.get("lo", 0), pr.get("hi", 0), pr.get("box", (0,) * 6),
                                pr.get("negate", False))
            assert n == len(ok), (pr, n, len(ok))
            _assert_same(p, gk, gv, ok, ov)
    finally:
        p.close()


@pytest.mark.parametrize("kind", (O.SET_U64, O.MAP_U64_U64))
def test_select_appends_and_counts_past_cap(kind):
    rng = np.random.default_rng(950 + kind)
    p = Pair(kind, 20000, bucket_bytes=64)
    try:
        keys = random_keys(kind, 10000, rng)
        p.insert(keys, value_for(kind, keys))
        half = 2**63
        # two selections appended to one output: the halves of the key space
        ko = torch.empty(12000, dtype=torch.int64, device="cuda")
        vo = torch.empty(12000, dtype=torch.int64, device="cuda") if p.is_map else None
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        p.g.select(L.PRED_KEY_RANGE, 0, half - 1, keys_out=ko, vals_out=vo if vo is not None else False, count=cnt)
        n1 = int(cnt.item())
        p.g.select(L.PRED_KEY_RANGE, half, 2**64 - 1, keys_out=ko, vals_out=vo if vo is not None else False, count=cnt)
        n = int(cnt.item())
        assert n == 10000 and 0 < n1 < n
        gk = to_numpy(ko[:n], np.uint64)
        assert (gk[:n1] < np.uint64(half)).all() and (gk[n1:] >= np.uint64(half)).all()
        ok, ov = p.o.dump()
        order = np.argsort(gk, kind="stable")
        C.assert_contents(gk[order], to_numpy(vo[:n], np.uint64)[order] if vo is not None else None, ok, ov)
        # an output of 1000 entries: all 10000 are counted, 1000 distinct stored keys are written
        small = torch.full((1000,), -1, dtype=torch.int64, device="cuda")
        cnt.zero_()
        p.g.select(L.PRED_ALL, keys_out=small, vals_out=False, count=cnt, cap=1000)
        assert int(cnt.item()) == 10000
        sk = to_numpy(small, np.uint64)
        assert len(np.unique(sk)) == 1000 and np.isin(sk, ok).all()
    finally:
        p.close()


def test_select_edges():
    """Empty table, zero capacity (count only), a predicate matching nothing,
    and a table holding only the two side-slot keys."""
    p = Pair(O.MAP_U64_U64, 1000, bucket_bytes=64)
    try:
        ko, vo, cnt = p.g.select(L.PRED_ALL, cap=0, keys_out=torch.empty(0, dtype=torch.int64, device="cuda"))
        assert int(cnt.item()) == 0
        keys = np.array(RESERVED[O.MAP_U64_U64])
        p.insert(keys, value_for(O.MAP_U64_U64, keys))
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        p.g.select(L.PRED_ALL, keys_out=torch.empty(0, dtype=torch.int64, device="cuda"), count=cnt, cap=0)
        assert int(cnt.item()) == 2                      # counted, nothing written
        gk, gv, n = _gpu_select(p, kind=L.PRED_ALL)
        ok, ov = p.o.select(O.PRED_ALL)
        _assert_same(p, gk, gv, ok, ov)
        gk, gv, n = _gpu_select(p, kind=L.PRED_KEY_RANGE, lo=0, hi=2**62)
        assert n == 0
    finally:
        p.close()
