"""Full-size workloads, in the launch configuration bench.py times, against
the CPU oracle.

* map<u64,u64> at 2^28 slots filled to load factor 0.8 in batches of 2^26
  (the bench's table and shapes): every insert status, the found flags and
  values of 2^26 present and 2^26 absent queries, every erase status, the
  size, and the sorted contents, before and after a rehash that purges the
  tombstones.
* The multi-table workload: all 1024 tables in the bench's tuned batched
  shape, table by table.

The oracle replays on the host (single-threaded per table; independent
tables on a thread pool, since its calls run without the interpreter lock)."""
import concurrent.futures as cf

import numpy as np
import pytest
import torch

import compare as C
from oracle import oracle as O
from paper_1908_05936_gb300 import _lib as L
from paper_1908_05936_gb300.table import Table, to_device, to_numpy
from workloads import recipes, splitmix

pytestmark = pytest.mark.gpu


def sorted_contents(t: Table):
    """The table's stored (keys, values) sorted by key bit pattern, sorted on
    the device (unsigned order: the sign bit flipped for the signed sort)."""
    k, v = t.dump()
    order = torch.argsort(k ^ torch.tensor(-(1 << 63), dtype=torch.int64, device=k.device))
    ks = to_numpy(k[order], np.uint64)
    vs = to_numpy(v[order], np.uint64) if v is not None else None
    return ks, vs


@pytest.mark.slow
def test_map_u64_2e28_lf08_against_oracle():
    from paper_1908_05936_gb300 import build
    build.build()
    slots, B = 1 << 28, 1 << 26
    n_fill = recipes.fill_count(slots, 0.8)
    fill = recipes.map_fill_keys(0, n_fill, 0)
    vals = splitmix.value_of(fill)
    hit = recipes.map_hit_keys(n_fill, B, 0)
    miss = recipes.map_miss_keys(B, 0, start=n_fill)
    er = recipes.map_hit_keys(n_fill, B, 0, salt=1)
    t = Table(L.MAP_U64_U64, slots, bucket_bytes=64)        # the bench's table, default launch shapes
    o = O.OracleTable(O.MAP_U64_U64, slots)
    with cf.ThreadPoolExecutor(1) as ex:                    # the oracle replays while the GPU runs
        fut = ex.submit(lambda: ([o.insert(fill[off:off + B], vals[off:off + B]) for off in range(0, n_fill, B)],
                                 o.find(hit), o.find(miss), o.erase(er), o.size()))
        gst = [to_numpy(t.insert(to_device(fill[off:off + B]), to_device(vals[off:off + B])), np.uint8)
               for off in range(0, n_fill, B)]
        gh = [to_numpy(x, np.uint8 if i == 0 else np.uint64) for i, x in enumerate(t.find(to_device(hit)))]
        gm = [to_numpy(x, np.uint8 if i == 0 else np.uint64) for i, x in enumerate(t.find(to_device(miss)))]
        ge = to_numpy(t.erase(to_device(er)), np.uint8)
        gsize = t.size()
        ost, oh, om, oe, osize = fut.result()
    for i, off in enumerate(range(0, n_fill, B)):
        C.assert_status(fill[off:off + B], gst[i], ost[i], f"insert batch {i}")
    C.assert_find(gh[0], gh[1], oh[0], oh[1], "find present")
    C.assert_find(gm[0], gm[1], om[0], om[1], "find absent")
    assert int(oh[0].sum()) == B and int(om[0].sum()) == 0
    C.assert_status(er, ge, oe, "erase")
    assert gsize == osize == n_fill - len(np.unique(er))
    gk, gv = sorted_contents(t)
    ok, ov = o.dump()
    C.assert_contents(gk, gv, ok, ov, "contents")
    t.rehash(slots)                                         # purges the tombstones, keeps the contents
    s = t.stats()
    assert s["live"] == s["used"] == osize
    gk, gv = sorted_contents(t)
    C.assert_contents(gk, gv, ok, ov, "contents after rehash")
    f, v = t.find(to_device(hit))
    of, ov2 = o.find(hit)
    C.assert_find(to_numpy(f, np.uint8), to_numpy(v, np.uint64), of, ov2, "find after rehash")
    t.close()
    o.close()


def _oracle_table(args):
    slots, ops = args
    orc = O.OracleTable(O.SET_U64, slots)
    res = orc.mixed(ops.insert_keys, None, ops.find_keys, ops.erase_keys)
    k, _ = orc.dump()
    orc.close()
    return res, k


@pytest.mark.slow
def test_multi_table_all_tables_against_oracle():
    """All 1024 tables of the batched workload (capacities log-uniform in
    2^10..2^22, 0.5 x capacity operations each: 60 % insert, 30 % find, 10 %
    erase), one graph launch in the bench's tuned shape, against the oracle's
    phase semantics table by table."""
    from paper_1908_05936_gb300 import build, tune
    from paper_1908_05936_gb300.batch import Batch, Item
    build.build()
    slots = recipes.multi_table_slots()
    n_tab = len(slots)
    assert n_tab == 1024
    ops = [recipes.multi_table_ops(int(slots[t]), t) for t in range(n_tab)]
    shape = tune.batch_config() or dict(bucket_bytes=128, lane_bytes=0, keys_per_group=0, block=0, tile=4096)
    with cf.ThreadPoolExecutor(16) as ex:
        fut = [ex.submit(_oracle_table, (int(slots[t]), ops[t])) for t in range(n_tab)]
        tabs, items, outs = [], [], []
        for t in range(n_tab):
            tab = Table(L.SET_U64, int(slots[t]), bucket_bytes=shape["bucket_bytes"])
            o = ops[t]
            ki, kf, ke = to_device(o.insert_keys), to_device(o.find_keys), to_device(o.erase_keys)
            si, ff, se = (torch.empty(x.numel(), dtype=torch.uint8, device="cuda") for x in (ki, kf, ke))
            items += [Item(tab, L.OP_INSERT, ki, None, si), Item(tab, L.OP_FIND, kf, None, ff),
                      Item(tab, L.OP_ERASE, ke, None, se)]
            tabs.append(tab)
            outs.append((si, ff, se))
        b = Batch(items, lane_bytes=shape["lane_bytes"], keys_per_group=shape["keys_per_group"], block=shape["block"],
                  tile=shape["tile"], use_graph=True)
        b.launch()
        torch.cuda.synchronize()
        total = 0
        for t in range(n_tab):
            (ist, (of, _), est), ok = fut[t].result()
            o = ops[t]
            si, ff, se = (to_numpy(x, np.uint8) for x in outs[t])
            C.assert_status(o.insert_keys, si, ist, f"table {t} insert")
            C.assert_find(ff, None, of, None, f"table {t} find")
            C.assert_status(o.erase_keys, se, est, f"table {t} erase")
            gk, _ = tabs[t].dump_numpy()
            C.assert_contents(gk, None, ok, None, f"table {t} contents")
            total += len(o.insert_keys) + len(o.find_keys) + len(o.erase_keys)
            tabs[t].close()
        b.close()
    assert total > 2 * 10**8                     # the whole workload (about 2.5e8 operations)


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
