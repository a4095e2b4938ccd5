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
    for t in sample:
        tab = Table(L.SET_U64, int(slots[t]), bucket_bytes=128)
        o = ops[t]
        ki, kf, ke = to_device(o.insert_keys), to_device(o.find_keys), to_device(o.erase_keys)
        si, ff, se = (torch.empty(x.numel(), dtype=torch.uint8, device="cuda") for x in (ki, kf, ke))
        items += [Item(tab, L.OP_INSERT, ki, None, si), Item(tab, L.OP_FIND, kf, None, ff),
                  Item(tab, L.OP_ERASE, ke, None, se)]
        tabs[t] = tab
        outs[t] = (si, ff, se)
    b = Batch(items, tile=4096, use_graph=True)
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
