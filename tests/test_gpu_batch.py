"""Batched form (one persistent launch per phase over many tables, optionally a
CUDA graph): every table's results equal the oracle's phase semantics and the
plain one-launch-per-call path run alone."""
import numpy as np
import pytest
import torch

import compare as C
from oracle import oracle as O
from paper_1908_05936_gb300 import _lib as L
from paper_1908_05936_gb300.batch import Batch, Item
from paper_1908_05936_gb300.table import Table, to_device, to_numpy
from workloads import recipes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1908_05936_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def make_tables(n_tables, lo, hi, seed=0, bucket_bytes=None):
    slots = recipes.multi_table_slots(n_tables, lo, hi, seed=seed)
    ops = [recipes.multi_table_ops(int(s), t, seed=seed) for t, s in enumerate(slots)]
    bbs = [bucket_bytes or (32, 64, 128)[t % 3] for t in range(n_tables)]
    return slots, ops, bbs


def build_items(tables, ops):
    items, outs = [], []
    for t, (tab, o) in enumerate(zip(tables, ops)):
        ki, kf, ke = to_device(o.insert_keys), to_device(o.find_keys), to_device(o.erase_keys)
        si = torch.empty(len(o.insert_keys), dtype=torch.uint8, device="cuda")
        ff = torch.empty(len(o.find_keys), dtype=torch.uint8, device="cuda")
        se = torch.empty(len(o.erase_keys), dtype=torch.uint8, device="cuda")
        items += [Item(tab, L.OP_INSERT, ki, out=si), Item(tab, L.OP_FIND, kf, out=ff),
                  Item(tab, L.OP_ERASE, ke, out=se)]
        outs.append((si, ff, se))
    return items, outs


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("lb,kpt", [(0, 1), (32, 2), (0, 2), (0, 4), (0, 8)])
def test_batched_equals_oracle_and_plain(graph, lb, kpt):
    slots, ops, bbs = make_tables(48, 10, 15, seed=1)
    tables = [Table(L.SET_U64, int(s), bucket_bytes=bb) for s, bb in zip(slots, bbs)]
    items, outs = build_items(tables, ops)
    b = Batch(items, lane_bytes=lb, keys_per_group=kpt, tile=512, use_graph=graph)
    for rep in range(2):                    # a replay re-applies the same calls
        b.launch()
        torch.cuda.synchronize()
        if rep == 0:
            oracles = [O.OracleTable(O.SET_U64, int(s)) for s in slots]
        for t, (o, orc) in enumerate(zip(ops, oracles)):
            ist, (ff, _), est = orc.mixed(o.insert_keys, None, o.find_keys, o.erase_keys)
            si, gf, se = (to_numpy(x, np.uint8) for x in outs[t])
            C.assert_status(o.insert_keys, si, ist, f"table {t} insert")
            C.assert_find(gf, None, ff, None, f"table {t} find")
            C.assert_status(o.erase_keys, se, est, f"table {t} erase")
    # plain path, same calls one table at a time
    for t, (o, orc) in enumerate(zip(ops, oracles)):
        gk, _ = tables[t].dump_numpy()
        ok, _ = orc.dump()
        C.assert_contents(gk, None, ok, None, f"table {t} contents")
        assert tables[t].size() == orc.size()
        plain = Table(L.SET_U64, int(slots[t]), bucket_bytes=bbs[t])
        for _ in range(2):
            si = plain.insert(to_device(o.insert_keys))
            f, _ = plain.find(to_device(o.find_keys))
            se = plain.erase(to_device(o.erase_keys))
        assert np.array_equal(to_numpy(f, np.uint8), to_numpy(outs[t][1], np.uint8))
        C.assert_status(o.erase_keys, to_numpy(se, np.uint8), to_numpy(outs[t][2], np.uint8))
        pk, _ = plain.dump_numpy()
        assert np.array_equal(pk, gk)
        plain.close()
    b.close()
    for tb in tables:
        tb.close()


@pytest.mark.parametrize("kpt", [1, 4])
def test_batched_maps_mixed_kinds(kpt):
    """Items of different kinds and ops in one batch: each phase runs one
    persistent launch per kind."""
    rng = np.random.default_rng(4)
    tabs, orcs, items, checks = [], [], [], []
    for kind in (O.SET_U32, O.SET_U64, O.MAP_I64_I32, O.MAP_U64_U64):
        slots = 5000
        t = Table(kind, slots, bucket_bytes=64)
        o = O.OracleTable(kind, slots)
        from gpu_pair import random_keys, value_for
        k = random_keys(kind, 3000, rng)
        v = value_for(kind, k)
        q = np.concatenate([k[:1000], random_keys(kind, 1000, rng)])
        e = k[::3]
        dk, dq, de = to_device(k), to_device(q), to_device(e)
        dv = to_device(v) if v is not None else None
        si = torch.empty(len(k), dtype=torch.uint8, device="cuda")
        ff = torch.empty(len(q), dtype=torch.uint8, device="cuda")
        fv = torch.empty(len(q), dtype=torch.int32 if kind == O.MAP_I64_I32 else torch.int64,
                         device="cuda") if v is not None else None
        se = torch.empty(len(e), dtype=torch.uint8, device="cuda")
        items += [Item(t, L.OP_INSERT, dk, dv, si), Item(t, L.OP_FIND, dq, None, ff, fv), Item(t, L.OP_ERASE, de, None, se)]
        tabs.append(t)
        orcs.append(o)
        checks.append((kind, k, v, q, e, si, ff, fv, se))
    b = Batch(items, lane_bytes=0, keys_per_group=kpt, tile=256, use_graph=True)
    b.launch()
    torch.cuda.synchronize()
    for o, (kind, k, v, q, e, si, ff, fv, se) in zip(orcs, checks):
        ist, (of, ov), est = o.mixed(k, v, q, e)
        C.assert_status(k, to_numpy(si, np.uint8), ist)
        C.assert_find(to_numpy(ff, np.uint8), to_numpy(fv, O.VAL_DTYPE[kind]) if fv is not None else None, of, ov)
        C.assert_status(e, to_numpy(se, np.uint8), est)
    b.close()
    for t in tabs:
        t.close()


def test_batch_tuner_sweeps_every_shape_and_its_choice_is_exact():
    """tune.py --batch on a small multi-table workload: one timing per bucket
    size and candidate shape, the fastest returned; the chosen shape (with
    its bucket size) then gives the oracle's results on another workload."""
    from paper_1908_05936_gb300 import tune
    rows = []
    best = tune.tune_batch(n_tables=12, buckets=(32, 64), reps=1, seed=5, save=False, every=rows)
    assert len(rows) == len(tune.batch_candidates(32)) + len(tune.batch_candidates(64))
    assert best["ms"] == min(r["ms"] for r in rows) and best["bucket_bytes"] in (32, 64)
    slots, ops, _ = make_tables(24, 10, 14, seed=6)
    tables = [Table(L.SET_U64, int(s), bucket_bytes=best["bucket_bytes"]) for s in slots]
    items, outs = build_items(tables, ops)
    b = Batch(items, lane_bytes=best["lane_bytes"], keys_per_group=best["keys_per_group"], block=best["block"],
              tile=best["tile"], use_graph=True)
    b.launch()
    torch.cuda.synchronize()
    for t, (o, s) in enumerate(zip(ops, slots)):
        orc = O.OracleTable(O.SET_U64, int(s))
        ist, (ff, _), est = orc.mixed(o.insert_keys, None, o.find_keys, o.erase_keys)
        si, gf, se = (to_numpy(x, np.uint8) for x in outs[t])
        C.assert_status(o.insert_keys, si, ist, f"table {t} insert")
        C.assert_find(gf, None, ff, None, f"table {t} find")
        C.assert_status(o.erase_keys, se, est, f"table {t} erase")
        gk, _ = tables[t].dump_numpy()
        ok, _ = orc.dump()
        C.assert_contents(gk, None, ok, None, f"table {t} contents")
    b.close()
    for tb in tables:
        tb.close()
