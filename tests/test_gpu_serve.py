"""Served form: every request's result in the mix (continuous batching,
merged launches, several lanes overlapping on the GPU, admission against a
scratch budget) equals the CPU oracle's result for that request when its
table's requests are replayed in arrival order, and equals the same requests
replayed alone through the plain GPU path.  Exact integer results; duplicate
keys inside one request compared as a multiset (compare.py)."""
import concurrent.futures as cf

import numpy as np
import pytest
import torch

import compare as C
from oracle import oracle as O
from paper_1908_05936_gb300 import _lib as L
from paper_1908_05936_gb300.serve import Server, ServedRequest
from paper_1908_05936_gb300.table import Table, to_numpy
from workloads import recipes, splitmix

pytestmark = pytest.mark.gpu


def make_tables(n_tables, slots, prefill, seed):
    tabs = []
    for t in range(n_tables):
        tab = Table(L.MAP_U64_U64, slots, bucket_bytes=128)
        k = splitmix.stream_u64(7000 + t, seed, 0, prefill)
        tab.insert(torch.from_numpy(k.view(np.int64)).cuda(),
                   torch.from_numpy(splitmix.value_of(k).view(np.int64)).cuda(), status=False)
        tabs.append(tab)
    torch.cuda.synchronize()
    return tabs


def make_requests(n_req, n_tables, rate, seed, max_log2=14):
    cdf = recipes.zipf_cdf(1 << 16)
    out = []
    for q in recipes.served_requests(n_req, n_tables, rate, seed=seed, max_log2=max_log2):
        keys = recipes.zipf_keys(q.table, q.key_stream, q.n, cdf, seed)
        kt = torch.from_numpy(keys.view(np.int64)).pin_memory()
        vt = torch.from_numpy(splitmix.value_of(keys).view(np.int64)).pin_memory() if q.op == 0 else None
        out.append(ServedRequest(q.rid, q.table, q.op, kt, vt, q.arrival))
    return out


@pytest.mark.parametrize("merge", [True, False])
def test_served_equals_alone(merge):
    from paper_1908_05936_gb300 import build
    build.build()
    n_tables, slots = 6, 1 << 18
    mix_tabs = make_tables(n_tables, slots, 1 << 16, seed=1)
    alone_tabs = make_tables(n_tables, slots, 1 << 16, seed=1)
    reqs = make_requests(240, n_tables, rate=20000.0, seed=3)
    srv = Server(mix_tabs, slot_bytes=1 << 20, lanes=3, merge=merge, depth=2, max_items=8)
    stats = srv.run(reqs, realtime=True)
    assert stats["requests"] == len(reqs)
    assert stats["launches"] == len(reqs) if not merge else stats["launches"] <= len(reqs)
    for r in sorted(reqs, key=lambda r: r.rid):
        t = alone_tabs[r.table]
        k = r.keys.cuda()
        if r.op == L.OP_INSERT:
            st = to_numpy(t.insert(k, r.vals.cuda()), np.uint8)
            C.assert_status(r.keys.numpy(), r.status, st, f"request {r.rid} insert")
        elif r.op == L.OP_FIND:
            f, v = t.find(k)
            C.assert_find(r.status, r.values, to_numpy(f, np.uint8), to_numpy(v, np.int64),
                          f"request {r.rid} find")
        else:
            st = to_numpy(t.erase(k), np.uint8)
            C.assert_status(r.keys.numpy(), r.status, st, f"request {r.rid} erase")
    for a, b in zip(mix_tabs, alone_tabs):
        ka, va = a.dump_numpy()
        kb, vb = b.dump_numpy()
        C.assert_contents(ka, va, kb, vb)
    for t in mix_tabs + alone_tabs:
        t.close()


def test_server_timeout_reports_and_recovers():
    """A run that cannot finish within its time limit returns HC_ERR_STATE
    after waiting for its launches; the same server then serves normally."""
    n_tables, slots = 2, 1 << 16
    tabs = make_tables(n_tables, slots, 1 << 12, seed=5)
    srv = Server(tabs, slot_bytes=1 << 20, lanes=2, merge=True, depth=2, max_items=4)
    reqs = make_requests(20, n_tables, rate=1e6, seed=6, max_log2=10)
    with pytest.raises(L.HCError):
        srv.run(reqs, realtime=True, timeout_s=0.0)
    stats = srv.run(make_requests(20, n_tables, rate=1e6, seed=7, max_log2=10), realtime=False)
    assert stats["requests"] == 20
    srv.close()
    for t in tabs:
        t.close()


def _oracle_replay(args):
    """One table's requests, in arrival order, through the oracle after the
    same prefill: the expected result of every request and the final
    contents."""
    slots, prefill_keys, reqs = args
    o = O.OracleTable(O.MAP_U64_U64, slots)
    o.insert(prefill_keys, splitmix.value_of(prefill_keys))
    out = {}
    for rid, op, keys, vals in reqs:
        if op == L.OP_INSERT:
            out[rid] = o.insert(keys, vals)
        elif op == L.OP_FIND:
            out[rid] = o.find(keys)
        else:
            out[rid] = o.erase(keys)
    k, v = o.dump()
    o.close()
    return out, (k, v)


@pytest.mark.slow
@pytest.mark.parametrize("merge", [True, False])
def test_served_against_oracle(merge):
    """A run shaped like the served workload (16 resident map<u64,u64>
    tables prefilled to load factor 0.5; Poisson arrivals of
    insert/find/erase requests 40/50/10 with sizes floor(2^U(0,20)) and
    Zipf(1.1) keys over 2^24 ranks per table; merged and one launch per
    request), against the oracle replaying each table's requests in arrival
    order: every request's statuses, found flags and values, and every
    table's final contents."""
    from paper_1908_05936_gb300 import build
    build.build()
    n_tables, slots = 16, 1 << 22
    prefill = slots // 2
    spec = recipes.served_requests(400, n_tables, 20000.0, seed=11, max_log2=20)
    cdf = recipes.zipf_cdf(1 << 24)
    keys = [recipes.zipf_keys(q.table, q.key_stream, q.n, cdf) for q in spec]
    pre = [splitmix.stream_u64(7000 + t, 0, 0, prefill) for t in range(n_tables)]
    per_table = [[] for _ in range(n_tables)]
    for q, k in zip(spec, keys):                   # spec is sorted by arrival
        per_table[q.table].append((q.rid, q.op, k, splitmix.value_of(k) if q.op == L.OP_INSERT else None))
    with cf.ThreadPoolExecutor(16) as ex:
        fut = [ex.submit(_oracle_replay, (slots, pre[t], per_table[t])) for t in range(n_tables)]
        tabs = []
        for t in range(n_tables):
            tab = Table(L.MAP_U64_U64, slots, bucket_bytes=64)
            tab.insert(torch.from_numpy(pre[t].view(np.int64)).cuda(),
                       torch.from_numpy(splitmix.value_of(pre[t]).view(np.int64)).cuda(), status=False)
            tabs.append(tab)
        torch.cuda.synchronize()
        reqs = []
        for q, k in zip(spec, keys):
            kt = torch.from_numpy(k.view(np.int64)).pin_memory()
            vt = torch.from_numpy(splitmix.value_of(k).view(np.int64)).pin_memory() if q.op == L.OP_INSERT else None
            reqs.append(ServedRequest(q.rid, q.table, q.op, kt, vt, q.arrival))
        srv = Server(tabs, lanes=4, depth=2, merge=merge)
        stats = srv.run(reqs, realtime=True)
        assert stats["requests"] == len(reqs) and stats["ops"] == sum(q.n for q in spec)
        expected = [f.result() for f in fut]
    for r in reqs:
        exp = expected[r.table][0][r.rid]
        if r.op == L.OP_FIND:
            C.assert_find(r.status, r.values.view(np.uint64), exp[0], exp[1], f"request {r.rid} find")
        else:
            C.assert_status(r.keys.numpy(), r.status, exp, f"request {r.rid} {'insert' if r.op == 0 else 'erase'}")
    for t in range(n_tables):
        gk, gv = tabs[t].dump_numpy()
        ok, ov = expected[t][1]
        C.assert_contents(gk, gv, ok, ov, f"table {t} contents")
    srv.close()
    for tab in tabs:
        tab.close()
