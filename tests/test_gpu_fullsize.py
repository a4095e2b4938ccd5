"""Full-size workloads, in the launch configuration bench.py times.

map<u64,u64> at 2^28 slots filled to load factor 0.8 in 2^26 batches is far
beyond what the CPU oracle replays in seconds, so it is checked by properties
that hold at any size and are exact: with distinct keys every insert reports
INSERTED and the size equals the fill; every present query finds its key with
the value splitmix64(key) it was inserted with; fresh keys are absent; an erase
of 2^26 present keys reports ERASED once per key and those keys are then absent;
a rehash keeps every key.  The multi-table workload (1024 tables) is compared
with the oracle table by table on a seeded sample of the tables."""
import numpy as np
import pytest
import torch

import compare as C
from oracle import oracle as O
from paper_1908_05936_gb300 import _lib as L
from paper_1908_05936_gb300.table import Table, to_device, to_numpy
from workloads import gpu as G
from workloads import recipes

pytestmark = pytest.mark.gpu


def test_map_u64_2e28_lf08_properties():
    from paper_1908_05936_gb300 import build
    build.build()
    slots, B = 1 << 28, 1 << 26
    n_fill = recipes.fill_count(slots, 0.8)
    t = Table(L.MAP_U64_U64, slots, bucket_bytes=64)
    st = torch.empty(B, dtype=torch.uint8, device="cuda")
    inserted = 0
    for off in range(0, n_fill, B):
        n = min(B, n_fill - off)
        k = G.stream_u64(3, 0, off, n)
        t.insert(k, G.value_of(k), status=st[:n])
        inserted += int((st[:n] == 0).sum())
    # 214,748,364 uniform 64-bit keys are distinct (a repeat has probability ~1e-3)
    assert inserted == n_fill and t.size() == n_fill
    hit = G.sample_u64(3, n_fill, B, 14, 0)
    f, v = t.find(hit)
    assert bool(f.all()) and bool((v == G.value_of(hit)).all())
    miss = G.stream_u64(4, 0, n_fill, B)
    f, _ = t.find(miss)
    assert int(f.sum()) == 0
    er = G.sample_u64(3, n_fill, B, 16, 0)
    t.erase(er, status=st)
    assert bool((st == L.ERASED).all()) and t.size() == n_fill - B
    f, _ = t.find(er)
    assert int(f.sum()) == 0
    t.rehash(slots)                                  # purge the tombstones
    s = t.stats()
    assert s["live"] == n_fill - B and s["used"] == n_fill - B
    f, v = t.find(hit)
    want = ~np.isin(to_numpy(hit, np.uint64), to_numpy(er, np.uint64))
    assert np.array_equal(to_numpy(f, np.uint8).astype(bool), want)
    t.close()


def test_multi_table_full_sampled_tables():
    from paper_1908_05936_gb300 import build
    from paper_1908_05936_gb300.batch import Batch, Item
    build.build()
    slots = recipes.multi_table_slots()
    rng = np.random.default_rng(0)
    sample = sorted(rng.choice(len(slots), size=24, replace=False).tolist())
    ops = {t: recipes.multi_table_ops(int(slots[t]), t) for t in sample}
    tabs, items, outs = {}, [], {}
    from paper_1908_05936_gb300 import tune
    # the shape bench.py times: the tuner's, else the untuned default
    shape = tune.batch_config() or dict(bucket_bytes=128, lane_bytes=0, keys_per_group=0, block=0, tile=4096)
    for t in sample:
        tab = Table(L.SET_U64, int(slots[t]), bucket_bytes=shape["bucket_bytes"])
        o = ops[t]
        ki, kf, ke = to_device(o.insert_keys), to_device(o.find_keys), to_device(o.erase_keys)
        si, ff, se = (torch.empty(x.numel(), dtype=torch.uint8, device="cuda") for x in (ki, kf, ke))
        items += [Item(tab, L.OP_INSERT, ki, None, si), Item(tab, L.OP_FIND, kf, None, ff),
                  Item(tab, L.OP_ERASE, ke, None, se)]
        tabs[t] = tab
        outs[t] = (si, ff, se)
    b = Batch(items, lane_bytes=shape["lane_bytes"], keys_per_group=shape["keys_per_group"], block=shape["block"],
              tile=shape["tile"], use_graph=True)
    b.launch()
    torch.cuda.synchronize()
    for t in sample:
        o = ops[t]
        orc = O.OracleTable(O.SET_U64, int(slots[t]))
        ist, (of, _), est = orc.mixed(o.insert_keys, None, o.find_keys, o.erase_keys)
        si, ff, se = (to_numpy(x, np.uint8) for x in outs[t])
        C.assert_status(o.insert_keys, si, ist, f"table {t} insert")
        C.assert_find(ff, None, of, None, f"table {t} find")
        C.assert_status(o.erase_keys, se, est, f"table {t} erase")
        gk, _ = tabs[t].dump_numpy()
        ok, _ = orc.dump()
        C.assert_contents(gk, None, ok, None, f"table {t} contents")
        orc.close()
        tabs[t].close()
    b.close()


def test_small_inserts_into_a_table_beyond_l2():
    """Inserts of 2^16 keys into a 256 MiB map run one key per thread in lock
    step (the small-insert rule); with in-batch duplicates, present keys and
    erases in between they match the oracle call by call."""
    import gpu_pair as GP
    rng = np.random.default_rng(2024)
    p = GP.Pair(O.MAP_U64_U64, 1 << 24, bucket_bytes=64)
    try:
        dom = GP.random_keys(O.MAP_U64_U64, 1 << 18, rng)
        for b in range(6):
            keys = dom[rng.integers(0, len(dom), size=1 << 16)]
            p.insert(keys, GP.value_for(O.MAP_U64_U64, keys, salt=b))
            p.find(dom[rng.integers(0, len(dom), size=1 << 15)])
            p.erase(keys[::5])
        p.check()
    finally:
        p.close()


def test_ordered_calls_at_scale():
    """Ordered insert and erase of 2^20 draws from 2^19 keys (each key about
    twice, equal keys with different values) on a 2^22-slot map, position by
    position against the sequential oracle."""
    rng = np.random.default_rng(2025)
    t = Table(L.MAP_U64_U64, 1 << 22, bucket_bytes=64)
    o = O.OracleTable(O.MAP_U64_U64, 1 << 22)
    try:
        dom = rng.integers(0, 2**63, size=1 << 19, dtype=np.int64).view(np.uint64)
        keys = dom[rng.integers(0, len(dom), size=1 << 20)]
        vals = rng.integers(0, 2**63, size=len(keys), dtype=np.int64).view(np.uint64)
        gs = to_numpy(t.insert_ordered(to_device(keys), to_device(vals)), np.uint8)
        assert np.array_equal(gs, o.insert(keys, vals))
        q = dom[rng.integers(0, len(dom), size=1 << 18)]
        gf, gv = t.find(to_device(q))
        of, ov = o.find(q)
        C.assert_find(to_numpy(gf, np.uint8), to_numpy(gv, np.uint64), of, ov)
        er = dom[rng.integers(0, len(dom), size=1 << 20)]
        ge = to_numpy(t.erase_ordered(to_device(er)), np.uint8)
        assert np.array_equal(ge, o.erase(er))
        gk, gvals = t.dump_numpy()
        ok, ov = o.dump()
        C.assert_contents(gk, gvals, ok, ov, "contents after ordered calls")
    finally:
        t.close()
        o.close()
