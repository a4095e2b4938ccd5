"""Autotuner of launch shapes (lane width = lanes per key, keys in flight,
block size) per container kind, operation and bucket size, on the current
GPU.  Results never depend on the shape; only speed does.

    python -m paper_1908_05936_gb300.tune [--kinds map_u64_u64,set_u64] [--slots-log2 26]

For each (kind, bucket bytes) it fills a table to load factor 0.8 in batches
of 2^(slots_log2 - 2) keys, then times every candidate shape on insert (the
last batch of the fill), find (all present), find (all absent) and erase
with CUDA events, and keeps the fastest shape per operation; "find" is the
shape with the least time for the present and the absent batch together,
the one `apply()` installs.  The winners are
written to a JSON cache keyed by device name and SM count
(`tuned.json` next to this file); `apply()` installs them on a table.

    python -m paper_1908_05936_gb300.tune --batch [--tables 1024]

tunes the batched form instead: on the multi-table workload (1024 set<u64>
tables with capacities log-uniform in 2^10..2^22, each given 0.5 x its
capacity in operations, 60 / 30 / 10 insert / find / erase) it times one
batched launch for every bucket size and launch shape (lane width, keys per
thread, block, keys per chunk) and caches the fastest as "batch/set_u64";
`batch_config()` returns it.
"""
from __future__ import annotations

import argparse
import json
import os

import torch

from . import _lib as L
from .table import KIND_NAMES, Table

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")
LANES = (16, 32, 64, 128)
KEYS_IN_FLIGHT = (1, 2)
BLOCKS = (64, 128, 256)


def device_key() -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}/{p.multi_processor_count}SM"


def _keys(kind: int, stream: int, start: int, n: int):
    from workloads import gpu as G
    if kind == L.SET_U32:
        return G.stream_u32(stream, 0, start, n)
    return G.stream_u64(stream, 0, start, n)


def _vals(kind: int, keys):
    from workloads import gpu as G
    if kind == L.MAP_U64_U64:
        return G.value_of(keys)
    if kind == L.MAP_I64_I32:
        return (G.value_of(keys) & 0x7FFFFFFF).to(torch.int32)
    return None


def _time(fn, reps: int = 3) -> float:
    s = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _time_once(fn) -> float:
    s = torch.cuda.current_stream()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s)
    fn()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def candidates(table: Table) -> list[dict]:
    krb = table.get_launch(0)["lane_bytes"]              # the bucket's key region
    lanes = [lb for lb in LANES if lb <= krb and (lb >= 32 or table.is_map)]
    if table.is_map:
        lanes.append(table.bucket_bytes)                  # keys and values in one read
    out = [dict(lane_bytes=lb, keys_per_group=k, block=b) for lb in lanes for k in KEYS_IN_FLIGHT for b in BLOCKS]
    # streaming forms: one thread per key over the key region, probes refilled as they finish
    out += [dict(lane_bytes=krb, keys_per_group=k, block=b) for k in (4, 8) for b in BLOCKS]
    # map lookups by lane pairs (one lane the keys, its partner the values)
    if table.is_map and 2 * krb == table.bucket_bytes:
        out += [dict(lane_bytes=table.bucket_bytes, keys_per_group=k, block=b, find_only=True) for k in (4, 8)
                for b in BLOCKS]
    return out


def tune_table(kind: int, bucket_bytes: int, slots_log2: int = 26, lf: float = 0.8, every: list | None = None) -> dict:
    """Best shape per operation; with `every` given, each candidate's timings
    are appended to it as well."""
    slots = 1 << slots_log2
    n_fill = int(lf * slots)
    batch = 1 << (slots_log2 - 2)
    t = Table(kind, slots, bucket_bytes=bucket_bytes)
    fill = _keys(kind, 3, 0, n_fill)
    vals = _vals(kind, fill)
    for off in range(0, n_fill - batch, batch):
        t.insert(fill[off:off + batch], vals[off:off + batch] if vals is not None else None, status=False)
    last = fill[n_fill - batch:]
    last_v = vals[n_fill - batch:] if vals is not None else None
    # present keys sampled from the whole fill (keys inserted early sit in
    # their first bucket more often than keys inserted at a high load factor)
    gen = torch.Generator(device="cuda").manual_seed(5)
    hit = fill[torch.randperm(n_fill, device="cuda", generator=gen)[:batch]]
    miss = _keys(kind, 4, 0, batch)
    out = torch.empty(batch, dtype=torch.uint8, device="cuda")
    vout = torch.empty(batch, dtype=torch.int32 if kind == L.MAP_I64_I32 else torch.int64, device="cuda") \
        if t.is_map else False
    results = {"insert": [], "find_hit": [], "find_miss": [], "erase": []}
    t.insert(last, last_v, status=False)                  # the table starts at the target load factor
    for c in candidates(t):
        find_only = c.pop("find_only", False)
        for op in ((L.OP_FIND,) if find_only else (L.OP_INSERT, L.OP_FIND, L.OP_ERASE)):
            t.set_launch(op, fold=2, **c)

        def ins():
            t.insert(last, last_v, status=out)

        def era():
            t.erase(last, status=out)

        # erase / re-insert the last batch: each insert stores new keys into a
        # table at the target load factor, each erase removes present keys
        if find_only:
            results["insert"].append((float("inf"), c))
            results["erase"].append((float("inf"), c))
        else:
            e_ms, i_ms = [], []
            for _ in range(2):
                e_ms.append(_time_once(era))
                i_ms.append(_time_once(ins))
            results["insert"].append((min(i_ms), c))
            results["erase"].append((min(e_ms), c))
        results["find_hit"].append((_time(lambda: t.find(hit, found=out, vals_out=vout)), c))
        results["find_miss"].append((_time(lambda: t.find(miss, found=out, vals_out=vout)), c))
    t.close()
    if every is not None:
        for i, (_, c) in enumerate(results["find_hit"]):
            row = dict(c, bucket_bytes=bucket_bytes, kind=kind)
            for op, lst in results.items():
                row[op + "_mops"] = round(batch / lst[i][0] / 1e3, 1) if lst[i][0] != float("inf") else None
            every.append(row)
    best = {}
    for op, lst in results.items():
        ms, c = min(lst, key=lambda x: x[0])
        best[op] = dict(c, ms=round(ms, 4), mops=round(batch / ms / 1e3, 1))
    # lookups of a mix of present and absent keys: the least total time
    both = [(h[0] + m[0], h[1]) for h, m in zip(results["find_hit"], results["find_miss"])]
    ms, c = min(both, key=lambda x: x[0])
    best["find"] = dict(c, ms=round(ms, 4), mops=round(2 * batch / ms / 1e3, 1))
    return best


def tune(kinds: list[int], buckets=(32, 64, 128), slots_log2: int = 26, save: bool = True,
         every: list | None = None) -> dict:
    res = {}
    for kind in kinds:
        name = [k for k, v in KIND_NAMES.items() if v == kind][0]
        for bb in buckets:
            res[f"{name}/{bb}"] = tune_table(kind, bb, slots_log2, every=every)
    if not save:
        return res
    cache = {}
    if os.path.exists(CACHE):
        with open(CACHE) as f:
            cache = json.load(f)
    cache.setdefault(device_key(), {}).update(res)
    with open(CACHE, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    return res


def apply(table: Table) -> bool:
    """Install the tuned shapes for this table's kind and bucket size on the
    current GPU, if the cache has them."""
    if not os.path.exists(CACHE):
        return False
    with open(CACHE) as f:
        cache = json.load(f).get(device_key(), {})
    name = [k for k, v in KIND_NAMES.items() if v == table.kind][0]
    best = cache.get(f"{name}/{table.bucket_bytes}")
    if not best:
        return False
    for op, key in ((L.OP_INSERT, "insert"), (L.OP_FIND, "find" if "find" in best else "find_hit"),
                    (L.OP_ERASE, "erase")):
        b = best[key]
        table.set_launch(op, lane_bytes=b["lane_bytes"], keys_per_group=b["keys_per_group"], block=b["block"])
    return True


def batch_candidates(bucket_bytes: int) -> list[dict]:
    """Launch shapes of the batched form for set<u64> tables of one bucket
    size: lock-step phases with one thread per key (lane 0) or 32-byte lanes,
    1 or 2 keys per thread; streaming phases with 4 keys per thread; blocks
    of 64 / 128 / 256 threads; chunks of 1024 or 4096 keys or the automatic
    size (0)."""
    lanes = (0, 32) if bucket_bytes > 32 else (0,)
    out = [dict(lane_bytes=lb, keys_per_group=k, block=b, tile=t)
           for lb in lanes for k in (1, 2) for b in (64, 128, 256) for t in (0, 1024, 4096)]
    out += [dict(lane_bytes=0, keys_per_group=4, block=b, tile=t) for b in (64, 128, 256) for t in (0, 1024, 4096)]
    return out


def tune_batch(n_tables: int = 1024, buckets=(32, 64, 128), reps: int = 3, seed: int = 0, save: bool = True,
               every: list | None = None) -> dict:
    """Time one batched launch of the multi-table workload for every bucket
    size and launch shape; every launch starts from cleared tables.  Returns
    (and caches) the fastest: bucket_bytes, the shape, ms and G ops/s."""
    from workloads import recipes

    from .batch import Batch, Item
    from .table import to_device
    slots = recipes.multi_table_slots(n_tables, seed=seed)
    ops = [recipes.multi_table_ops(int(sl), t, seed) for t, sl in enumerate(slots)]
    n_ops = sum(len(o.insert_keys) + len(o.find_keys) + len(o.erase_keys) for o in ops)
    dev = [(to_device(o.insert_keys), to_device(o.find_keys), to_device(o.erase_keys)) for o in ops]
    outs = [tuple(torch.empty(k.numel(), dtype=torch.uint8, device="cuda") for k in d) for d in dev]
    rows = []
    for bb in buckets:
        tabs = [Table(L.SET_U64, int(sl), bucket_bytes=bb) for sl in slots]
        items = []
        for t, (ki, kf, ke), (si, sf, se) in zip(tabs, dev, outs):
            items += [Item(t, L.OP_INSERT, ki, None, si), Item(t, L.OP_FIND, kf, None, sf),
                      Item(t, L.OP_ERASE, ke, None, se)]
        for c in batch_candidates(bb):
            batch = Batch(items, use_graph=True, **c)
            times = []
            for _ in range(reps + 1):
                for t in tabs:
                    t.clear()
                times.append(_time_once(batch.launch))
            batch.close()
            ms = sorted(times[1:])[len(times[1:]) // 2]          # median of the timed launches
            row = dict(c, bucket_bytes=bb, ms=round(ms, 4), mops=round(n_ops / ms / 1e3, 1))
            rows.append(row)
            if every is not None:
                every.append(row)
        for t in tabs:
            t.close()
        del items
        torch.cuda.empty_cache()
    best = dict(min(rows, key=lambda r: r["ms"]), tables=n_tables, ops=n_ops)
    if save:
        cache = {}
        if os.path.exists(CACHE):
            with open(CACHE) as f:
                cache = json.load(f)
        cache.setdefault(device_key(), {})["batch/set_u64"] = best
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return best


def batch_config() -> dict | None:
    """The tuned batched-form shape for set<u64> tables on the current GPU
    (bucket_bytes, lane_bytes, keys_per_group, block, tile), or None."""
    if not os.path.exists(CACHE):
        return None
    with open(CACHE) as f:
        best = json.load(f).get(device_key(), {}).get("batch/set_u64")
    if not best:
        return None
    return {k: best[k] for k in ("bucket_bytes", "lane_bytes", "keys_per_group", "block", "tile")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", action="store_true", help="tune the batched form on the multi-table workload")
    ap.add_argument("--tables", type=int, default=1024)
    ap.add_argument("--kinds", default="map_u64_u64,set_u64,set_u32,map_i64_i32")
    ap.add_argument("--buckets", default="32,64,128")
    ap.add_argument("--slots-log2", type=int, default=26)
    ap.add_argument("--all", action="store_true", help="also print every candidate's rates, one JSON line each")
    ap.add_argument("--no-save", action="store_true", help="leave the cache file unchanged")
    a = ap.parse_args()
    from . import build
    build.build()
    every = [] if a.all else None
    if a.batch:
        best = tune_batch(a.tables, tuple(int(b) for b in a.buckets.split(",")), save=not a.no_save, every=every)
        for row in every or []:
            print(json.dumps(row))
        print(json.dumps(best))
        return
    kinds = [KIND_NAMES[k] for k in a.kinds.split(",")]
    best = tune(kinds, tuple(int(b) for b in a.buckets.split(",")), a.slots_log2, save=not a.no_save, every=every)
    for row in every or []:
        print(json.dumps(row))
    print(json.dumps(best))


if __name__ == "__main__":
    main()
