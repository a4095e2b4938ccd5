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
@pytest.mark.parametrize("inputs", ["pinned", "mixed"])
@pytest.mark.parametrize("merge", [True, False])
def test_served_against_oracle(merge, inputs):
    """A run shaped like the served workload (16 resident map<u64,u64>
    tables prefilled to load factor 0.5; Poisson arrivals of
    insert/find/erase requests 40/50/10 with sizes floor(2^U(0,20)) and
    Zipf(1.1) keys over 2^24 ranks per table; merged and one launch per
    request), against the oracle replaying each table's requests in arrival
    order: every request's statuses, found flags and values, and every
    table's final contents.  Page-locked inputs run where they are; with
    "mixed" every other request's inputs are pageable and go through the
    slots' staging, so merged launches hold both kinds."""
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
        for i, (q, k) in enumerate(zip(spec, keys)):
            pin = inputs == "pinned" or i % 2 == 0
            kt = torch.from_numpy(k.view(np.int64).copy())
            vt = torch.from_numpy(splitmix.value_of(k).view(np.int64)) if q.op == L.OP_INSERT else None
            if pin:
                kt = kt.pin_memory()
                vt = vt.pin_memory() if vt is not None else None
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


def _expected(slots, pre, reqs_by_table):
    with cf.ThreadPoolExecutor(16) as ex:
        return list(ex.map(_oracle_replay, [(slots, pre[t], reqs_by_table[t]) for t in range(len(pre))]))


def _check_against(reqs, expected, tabs):
    for r in reqs:
        if r.rc != L.OK:
            continue
        exp = expected[r.table][0][r.rid]
        if r.op == L.OP_FIND:
            C.assert_find(r.status, r.values, exp[0], exp[1], f"request {r.rid} find")
        else:
            C.assert_status(r.keys.numpy(), r.status, exp, f"request {r.rid} op {r.op}")
    for t, tab in enumerate(tabs):
        gk, gv = tab.dump_numpy()
        ok, ov = expected[t][1]
        C.assert_contents(gk, gv, ok, ov, f"table {t} contents")


@pytest.mark.parametrize("merge", [True, False])
def test_live_submissions_from_two_threads_against_oracle(merge):
    """The server's own loop (hc_server_start) fed by two host threads at once
    (each submitting the requests of its own half of the tables, so a table's
    arrival order is its thread's order), with requests up to 5x a launch
    slot (cut into chunks); every result and the final contents against the
    oracle's replay of each table in that order.  Every other request has
    pageable inputs, so those go through the slots' staging (and the large
    ones are cut into chunks) while the page-locked ones run in place."""
    import threading
    from paper_1908_05936_gb300 import build
    build.build()
    n_tables, slots, prefill = 8, 1 << 20, 1 << 19
    spec = recipes.served_requests(160, n_tables, 1.0, seed=21, max_log2=17)
    cdf = recipes.zipf_cdf(1 << 20)
    pre = [splitmix.stream_u64(7100 + t, 0, 0, prefill) for t in range(n_tables)]
    tabs = []
    for t in range(n_tables):
        tab = Table(L.MAP_U64_U64, slots, bucket_bytes=64)
        tab.insert(torch.from_numpy(pre[t].view(np.int64)).cuda(),
                   torch.from_numpy(splitmix.value_of(pre[t]).view(np.int64)).cuda(), status=False)
        tabs.append(tab)
    torch.cuda.synchronize()
    reqs, per_table = [], [[] for _ in range(n_tables)]
    for i, q in enumerate(spec):
        k = recipes.zipf_keys(q.table, q.key_stream, q.n, cdf)
        v = splitmix.value_of(k) if q.op == L.OP_INSERT else None
        kt = torch.from_numpy(k.view(np.int64).copy())
        vt = torch.from_numpy(v.view(np.int64).copy()) if v is not None else None
        if i % 2 == 0:
            kt = kt.pin_memory()
            vt = vt.pin_memory() if vt is not None else None
        reqs.append(ServedRequest(q.rid, q.table, q.op, kt, vt))
        per_table[q.table].append((q.rid, q.op, k, v))
    srv = Server(tabs, slot_bytes=1 << 19, lanes=4, depth=2, merge=merge, max_items=8)
    # some pageable requests need several slots
    assert max(q.n for i, q in enumerate(spec) if i % 2) * 25 > 5 * (1 << 19)
    srv.start()
    errors = []

    def feed(parity):
        try:
            mine = [r for r in reqs if r.table % 2 == parity]
            for i, r in enumerate(mine):
                srv.submit(r)
                if i % 7 == 6:
                    srv.wait(mine[i - 3])                      # interleave waiting with submitting
        except Exception as e:                                 # reported by the main thread
            errors.append(e)

    th = [threading.Thread(target=feed, args=(p,)) for p in (0, 1)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    for r in reqs:
        assert srv.wait(r) == L.OK and r.rc == L.OK
    stats = srv.stop()
    assert stats["requests"] == len(reqs) and stats["timed_out"] == 0
    _check_against(reqs, _expected(slots, pre, per_table), tabs)
    srv.close()
    for tab in tabs:
        tab.close()


def test_deadline_drops_only_the_late_request():
    """One slot per lane, busy with a large request cut into many chunks;
    requests with a short deadline queued behind it on the same table are
    dropped (HC_ERR_TIMEOUT, nothing of them runs), the others are served,
    and everything that ran matches the oracle."""
    from paper_1908_05936_gb300 import build
    build.build()
    slots = 1 << 22
    pre = [splitmix.stream_u64(7200, 0, 0, 1 << 20)]
    tab = Table(L.MAP_U64_U64, slots, bucket_bytes=64)
    tab.insert(torch.from_numpy(pre[0].view(np.int64)).cuda(),
               torch.from_numpy(splitmix.value_of(pre[0]).view(np.int64)).cuda(), status=False)
    torch.cuda.synchronize()

    def req(rid, op, keys, deadline=0.0, pin=True):
        v = splitmix.value_of(keys) if op == L.OP_INSERT else None
        kt = torch.from_numpy(keys.view(np.int64).copy())
        vt = torch.from_numpy(v.view(np.int64).copy()) if v is not None else None
        if pin:
            kt = kt.pin_memory()
            vt = vt.pin_memory() if vt is not None else None
        return ServedRequest(rid, 0, op, kt, vt, deadline=deadline)

    # pageable inputs: staged through the slot, about 50 chunks of 1 MiB
    big = req(0, L.OP_INSERT, splitmix.stream_u64(7201, 0, 0, 1 << 21), pin=False)
    late = [req(1 + i, L.OP_INSERT, splitmix.stream_u64(7300 + i, 0, 0, 1000), deadline=1e-4) for i in range(3)]
    calm = req(4, L.OP_FIND, np.concatenate([pre[0][:500], late[0].keys.numpy().view(np.uint64)[:500]]))
    srv = Server([tab], slot_bytes=1 << 20, lanes=1, depth=1, merge=True)
    srv.start()
    for r in [big] + late + [calm]:
        srv.submit(r)
    assert srv.wait(big) == L.OK
    for r in late:
        assert srv.wait(r) == L.ERR_TIMEOUT and r.rc == L.ERR_TIMEOUT
    assert srv.wait(calm) == L.OK
    stats = srv.stop()
    assert stats["timed_out"] == 3 and stats["requests"] == 2
    per_table = [[(r.rid, r.op, r.keys.numpy().view(np.uint64), splitmix.value_of(r.keys.numpy().view(np.uint64))
                   if r.op == L.OP_INSERT else None) for r in (big, calm)]]
    exp = _expected(slots, pre, per_table)
    _check_against([big, calm] + late, exp, [tab])
    assert int(calm.status[500:].sum()) == 0                     # the dropped inserts never reached the table
    srv.close()
    tab.close()
