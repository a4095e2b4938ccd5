"""GPU containers against the CPU oracle, through the C ABI (parity tests).

Exact integer semantics: every comparison is bit-exact under the rules in
compare.py (duplicate keys inside one batch compared as a multiset)."""
import numpy as np
import pytest
import torch

import compare as C
from gpu_pair import RESERVED, Pair, edge_keys, random_keys, value_for
from paper_1908_05936_gb300.table import to_device, to_numpy
from oracle import oracle as O

pytestmark = pytest.mark.gpu

KINDS = (O.SET_U32, O.SET_U64, O.MAP_I64_I32, O.MAP_U64_U64)
SHAPES = [  # (bucket bytes, lane width, keys per group, block, fold); lane widths are
    # resolved per kind: wide = the whole key region, mid = half, narrow = 16 B (maps) / 32 B (sets),
    # full = the whole bucket, keys and values (maps; the key region for sets)
    (32, "wide", 1, 256, 1), (32, "wide", 2, 128, 2), (64, "wide", 1, 64, 1), (64, "narrow", 2, 256, 2),
    (64, "wide", 2, 256, 1), (128, "wide", 1, 128, 1), (128, "narrow", 2, 96, 2), (128, "mid", 1, 256, 1),
    (128, "wide", 2, 256, 2), (64, "full", 1, 128, 1), (128, "full", 2, 64, 2),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1908_05936_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield
    torch.cuda.synchronize()


def run_script(kind, slots, shape, seed, n_batches=30, domain_size=3000, max_batch=5000, rehash=True):
    bb, lb, kpt, block, fold = shape
    rng = np.random.default_rng(seed)
    dom = np.concatenate([random_keys(kind, domain_size, rng), edge_keys(kind)])
    p = Pair(kind, slots, bucket_bytes=bb, seed=seed,
             shape=dict(lane_bytes=lb, keys_per_group=kpt, block=block, fold=fold))
    try:
        for b in range(n_batches):
            op = rng.choice(["I", "I", "F", "E", "R", "C"] if rehash else ["I", "I", "F", "E"])
            n = int(rng.integers(0, max_batch))
            keys = random_keys(kind, n, rng, dom)
            if op == "I":
                p.insert(keys, value_for(kind, keys, salt=b))
            elif op == "F":
                p.find(keys)
            elif op == "E":
                p.erase(keys)
            elif op == "R":
                p.rehash(int(rng.integers(domain_size + 2, 2 * slots)))
            elif op == "C" and rng.random() < 0.3:
                p.clear()
            if b % 7 == 0:
                p.check()
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("shape", SHAPES, ids=[f"bb{s[0]}-lb{s[1]}-k{s[2]}-b{s[3]}-f{s[4]}" for s in SHAPES])
def test_random_scripts(kind, shape):
    run_script(kind, 4096, shape, seed=hash((kind, shape)) % 1000)


@pytest.mark.parametrize("kind", KINDS)
def test_batch_sizes_and_duplicates(kind):
    rng = np.random.default_rng(7)
    p = Pair(kind, 1 << 14)
    try:
        for n in (0, 1, 31, 32, 33, 127, 128, 129, 4097):
            keys = random_keys(kind, n, rng)
            p.insert(keys, value_for(kind, keys, salt=n))
            p.find(keys)
        p.check()
        # one key repeated across a whole batch: exactly one INSERTED
        k = np.full(4097, random_keys(kind, 1, rng)[0])
        gs, _ = p.insert(k, value_for(kind, k, salt=1))
        assert (gs == C.INSERTED).sum() == 1 and (gs == C.EXISTS).sum() == 4096
        gs, _ = p.erase(k)
        assert (gs == C.ERASED).sum() == 1
        # reserved bit patterns are ordinary keys
        r = np.array(list(RESERVED[kind]) * 40, dtype=O.KEY_DTYPE[kind])
        p.insert(r, value_for(kind, r, salt=2))
        p.find(r)
        p.check()
        p.erase(r)
        p.find(r)
        p.check()
        # keys not 16-byte aligned (scalar load path) and odd lengths
        keys = random_keys(kind, 1001, rng)
        dk = torch.from_numpy(keys.view(np.int32 if kind == O.SET_U32 else np.int64)).cuda()
        st = p.g.insert(dk[1:], None if not p.is_map else torch.from_numpy(
            value_for(kind, keys[1:]).view(np.int32 if kind == O.MAP_I64_I32 else np.int64)).cuda())
        ost = p.o.insert(keys[1:], value_for(kind, keys[1:]))
        C.assert_status(keys[1:], st.cpu().numpy(), ost)
        p.find(keys)
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bb", (32, 64, 128))
@pytest.mark.parametrize("slots", (1, 3, 17, 64, 1000))
def test_overflow_and_capacity(kind, bb, slots):
    """Fill past the capacity: the only failure, reported per key and as a
    sticky status; capacity is exact even when it is not a bucket multiple."""
    rng = np.random.default_rng(slots + bb)
    p = Pair(kind, slots, bucket_bytes=bb)
    res = {int(x) for x in C.bits(np.array(RESERVED[kind]))}
    try:
        keys = np.concatenate([random_keys(kind, slots + 5, rng), np.array(RESERVED[kind])])
        keys = np.concatenate([keys, keys[: len(keys) // 2]])          # duplicates too
        rng.shuffle(keys)
        vals = value_for(kind, keys)
        gs, _ = p.insert(keys, vals, check=False)
        gk, gv = p.g.dump_numpy()
        C.check_overflow_insert(keys, gs, set(), slots, {int(x) for x in C.bits(gk)}, res)
        assert p.g.size() == slots + 2
        from paper_1908_05936_gb300 import _lib as L
        assert p.g.status() == L.ERR_OVERFLOW
        assert p.g.status() == L.OK
        # stored values are the ones inserted with each stored key
        if p.is_map:
            f, v = p.g.find(torch.from_numpy(gk.view(np.int32 if kind == O.SET_U32 else np.int64)).cuda())
            assert f.all()
        # erase one stored key: exactly one more insert fits
        victim = gk[:1]
        assert p.g.erase(torch.from_numpy(victim.view(np.int64 if victim.dtype.itemsize == 8 else np.int32)).cuda()).cpu().numpy()[0] == C.ERASED
        more = random_keys(kind, 3, rng)
        st = p.g.insert(torch.from_numpy(more.view(np.int64 if more.dtype.itemsize == 8 else np.int32)).cuda(),
                        None if not p.is_map else torch.from_numpy(value_for(kind, more).view(
                            np.int32 if kind == O.MAP_I64_I32 else np.int64)).cuda()).cpu().numpy()
        assert sorted(st.tolist()) == [C.INSERTED, C.OVERFLOW, C.OVERFLOW]
    finally:
        p.close()


@pytest.mark.parametrize("kind", KINDS)
def test_rehash_clear_and_reinsert(kind):
    rng = np.random.default_rng(11)
    p = Pair(kind, 2048, bucket_bytes=64)
    try:
        keys = random_keys(kind, 1500, rng)
        p.insert(keys, value_for(kind, keys))
        p.erase(keys[:700])
        p.check()
        live_regular = p.o.size_regular()
        assert p.rehash(2048)               # same size: purges tombstones
        st = p.g.stats()
        assert st["used"] == live_regular and st["live"] == p.o.size()
        assert p.rehash(4000)
        assert not p.rehash(live_regular - 1)
        assert p.rehash(live_regular)       # exactly full
        p.check()
        more = random_keys(kind, 10, rng)
        gs, _ = p.insert(more, value_for(kind, more), check=False)
        assert (gs == C.OVERFLOW).all()
        p.rehash(5000)
        p.insert(keys[:700], value_for(kind, keys[:700]))   # erase then re-insert
        p.find(keys)
        p.check()
        p.clear()
        p.check()
        p.insert(keys, value_for(kind, keys))
        p.check()
    finally:
        p.close()


def test_set_u32_workload_full():
    """set<u32>, 2^21 slots: insert 1M uniform keys, find 1M (half present),
    erase 500k, all bit-exact against the oracle."""
    from workloads import recipes
    w = recipes.set_u32_workload()
    p = Pair(O.SET_U32, w.slots)
    try:
        p.insert(w.insert_keys)
        assert p.g.size() == len(np.unique(w.insert_keys))
        p.find(w.find_keys)
        p.erase(w.erase_keys)
        p.find(w.find_keys)
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("bb,lb,kpt", [(32, "wide", 1), (64, "wide", 1), (64, "full", 1), (128, "narrow", 2),
                                       (128, "wide", 1)])
def test_map_u64_load_factor_sweep_scaled(bb, lb, kpt):
    """map<u64,u64> at 2^20 slots: fill to 0.5/0.7/0.8/0.9 in batches, find
    2^16 present and 2^16 absent keys at each step, erase 2^16, contents."""
    from workloads import recipes
    slots = 1 << 20
    p = Pair(O.MAP_U64_U64, slots, bucket_bytes=bb,
             shape=dict(lane_bytes=lb, keys_per_group=kpt))
    try:
        done = 0
        for lf in (0.5, 0.7, 0.8, 0.9):
            target = recipes.fill_count(slots, lf)
            while done < target:
                n = min(1 << 16, target - done)
                k = recipes.map_fill_keys(done, n)
                p.insert(k, value_for(O.MAP_U64_U64, k))
                done += n
            p.find(recipes.map_hit_keys(done, 1 << 16))
            p.find(recipes.map_miss_keys(1 << 16, start=done))
        p.erase(recipes.map_hit_keys(done, 1 << 16, salt=1))
        p.find(recipes.map_hit_keys(done, 1 << 16))
        p.check()
    finally:
        p.close()


def test_teschner_hash_and_seeds_do_not_change_results():
    """Results are independent of the hash function and its seed."""
    rng = np.random.default_rng(3)
    xyz = rng.integers(-50, 50, size=(20000, 3))
    m = (1 << 21) - 1
    keys = ((xyz[:, 0] & m) | ((xyz[:, 1] & m) << 21) | ((xyz[:, 2] & m) << 42)).astype(np.int64)
    vals = value_for(O.MAP_I64_I32, keys)
    outs = []
    for hm, seed in ((0, 0), (0, 12345), (1, 0)):
        p = Pair(O.MAP_I64_I32, 30011, hash_mode=hm, seed=seed)
        try:
            p.insert(keys[:15000], vals[:15000])
            f, v = p.find(keys)
            p.erase(keys[::3])
            p.check()
            outs.append((f, v))
        finally:
            p.close()
    for f, v in outs[1:]:
        assert np.array_equal(f, outs[0][0]) and np.array_equal(v, outs[0][1])


def _pinned(a: np.ndarray) -> np.ndarray:
    """A page-locked copy of `a` with the same dtype."""
    out = torch.empty(a.nbytes, dtype=torch.uint8).pin_memory().numpy().view(a.dtype)   # the array keeps the tensor
    out[:] = a
    return out


@pytest.mark.parametrize("kind", (O.SET_U32, O.MAP_U64_U64))
@pytest.mark.parametrize("pinned", (False, True))
def test_host_buffer_calls(kind, pinned):
    """hc_*_host: host arrays in, host results out; pageable arrays go through
    chunked staging (two chunks here), page-locked ones are read and written
    in place by the kernels; same results as the oracle."""
    rng = np.random.default_rng(5)
    n = (1 << 22) + 12345
    p = Pair(kind, 1 << 24)
    host = _pinned if pinned else (lambda a: a)
    try:
        keys = random_keys(kind, n, rng)
        vals = value_for(kind, keys)
        st = host(np.empty(n, np.uint8))
        p.g.insert_host(host(keys), host(vals) if vals is not None else None, st)
        C.assert_status(keys, st, p.o.insert(keys, vals))
        q = np.concatenate([keys[: n // 2], random_keys(kind, n // 2, rng)])
        f = host(np.empty(len(q), np.uint8))
        v = host(np.empty(len(q), O.VAL_DTYPE[kind])) if kind in O.VAL_DTYPE else None
        p.g.find_host(host(q), f, v)
        of, ov = p.o.find(q)
        C.assert_find(f, v, of, ov)
        es = host(np.empty(len(keys[::2]), np.uint8))
        p.g.erase_host(host(np.ascontiguousarray(keys[::2])), es)
        C.assert_status(keys[::2], es, p.o.erase(keys[::2]))
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bb", (32, 64, 128))
@pytest.mark.parametrize("kpt", (4, 8))
@pytest.mark.parametrize("pair", (False, True))
def test_streaming_find(kind, bb, kpt, pair):
    """Streaming lookup (keys staged per block, several probes in flight per
    thread, refilled as they finish) against the oracle, with side-slot keys,
    duplicates, ragged chunk tails, absent and erased keys; for maps also by
    lane pairs (one lane reads the keys, its partner the values)."""
    if pair and kind not in (O.MAP_I64_I32, O.MAP_U64_U64):
        pytest.skip("lane pairs split map buckets")
    rng = np.random.default_rng(bb + kpt + kind)
    p = Pair(kind, 20000, bucket_bytes=bb)
    krb = p.g.get_launch(0)["lane_bytes"]
    p.g.set_launch(1, lane_bytes=bb if pair else krb, keys_per_group=kpt, block=96)
    try:
        keys = random_keys(kind, 15000, rng)
        keys = np.concatenate([keys, np.array(RESERVED[kind])])
        p.insert(keys, value_for(kind, keys))
        p.erase(keys[::5])
        for n in (0, 1, 95, 96, 97, 96 * kpt + 1, 40001):
            q = np.concatenate([keys, random_keys(kind, 30000, rng)])[rng.integers(0, 45002, size=n)]
            p.find(q)
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bb", (32, 64, 128))
@pytest.mark.parametrize("kpt", (4, 8))
def test_streaming_insert(kind, bb, kpt):
    """Streaming insert against the oracle: duplicates inside a batch,
    side-slot keys, tombstone reuse after erases, ragged chunk tails, the
    find-then-insert skip path, and overflow of a small table (invariants)."""
    rng = np.random.default_rng(100 + bb + kpt + kind)
    p = Pair(kind, 6000, bucket_bytes=bb)
    krb = p.g.get_launch(0)["lane_bytes"]
    p.g.set_launch(0, lane_bytes=krb, keys_per_group=kpt, block=64)
    dom = np.concatenate([random_keys(kind, 5000, rng), edge_keys(kind)])
    try:
        for b, n in enumerate((0, 1, 63, 64, 65, 64 * kpt + 3, 3000, 3000)):
            keys = dom[rng.integers(0, len(dom), size=n)]
            p.insert(keys, value_for(kind, keys, salt=b))
            p.erase(keys[::3])
        p.check()
        # find-then-insert: flagged keys are EXISTS without a probe
        keys = dom[rng.integers(0, len(dom), size=4000)]
        dk = to_device(keys)
        f, _ = p.g.find(dk, vals_out=False)
        st = to_numpy(p.g.insert_if_absent(dk, to_device(value_for(kind, keys)) if p.is_map else None, f), np.uint8)
        of, _ = p.o.find(keys)
        ost = np.full(len(keys), C.EXISTS, np.uint8)
        miss = np.nonzero(of == 0)[0]
        ost[miss] = p.o.insert(keys[miss], value_for(kind, keys)[miss] if p.is_map else None)
        C.assert_status(keys, st, ost, "insert_if_absent")
        p.check()
    finally:
        p.close()
    # overflow: a table of 100 slots takes 100 regular keys, the rest overflow
    q = Pair(kind, 100, bucket_bytes=bb)
    q.g.set_launch(0, lane_bytes=krb, keys_per_group=kpt, block=64)
    try:
        keys = random_keys(kind, 300, rng)
        gs, _ = q.insert(keys, value_for(kind, keys), check=False)
        gk, _ = q.g.dump_numpy()
        C.check_overflow_insert(keys, gs, set(), 100, {int(x) for x in C.bits(gk)}, set())
    finally:
        q.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bb", (32, 64, 128))
@pytest.mark.parametrize("kpt", (4, 8))
def test_streaming_erase(kind, bb, kpt):
    """Streaming erase against the oracle, with streaming insert and find on
    the same table: equal keys inside one erase call (one ERASED, the rest
    NOT_FOUND), side-slot keys, absent and already erased keys, ragged chunk
    tails, and re-inserts into the freed tombstones."""
    rng = np.random.default_rng(300 + bb + kpt + kind)
    p = Pair(kind, 8000, bucket_bytes=bb)
    krb = p.g.get_launch(0)["lane_bytes"]
    for op in (0, 1, 2):
        p.g.set_launch(op, lane_bytes=krb, keys_per_group=kpt, block=128)
    dom = np.concatenate([random_keys(kind, 7000, rng), edge_keys(kind)])
    try:
        p.insert(dom[:6000], value_for(kind, dom[:6000]))
        for b, n in enumerate((0, 1, 127, 128, 129, 128 * kpt + 5, 2500, 5000)):
            keys = dom[rng.integers(0, len(dom), size=n)]
            p.erase(keys)
            p.find(dom[rng.integers(0, len(dom), size=1000)])
            back = dom[rng.integers(0, len(dom), size=n // 2)]
            p.insert(back, value_for(kind, back, salt=b))
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("kind", KINDS)
def test_tombstone_reuse_keeps_keys_unique(kind):
    """Tiny tables: after an erase, a new key may land in the freed tombstone
    while a later slot of its bucket stays EMPTY; inserting it again must find
    it (EXISTS, stored once), a full table overflows, and clear frees it."""
    rng = np.random.default_rng(2000 + kind)
    for trial in range(40):
        p = Pair(kind, 4, bucket_bytes=32)
        try:
            keys = random_keys(kind, 8, rng)
            p.insert(keys[:3], value_for(kind, keys[:3]))
            p.erase(keys[:1])
            for k in (keys[3:5], keys[3:5], keys[:1], keys[3:6]):
                p.insert(k, value_for(kind, k))
            p.check()
            p.clear()
            p.insert(keys, value_for(kind, keys), check=False)
            assert p.g.size() == min(4, len(set(C.bits(keys).tolist())))
        finally:
            p.close()


def test_binding_refuses_short_buffers():
    """The kernels write outputs by index, so the binding refuses an output
    (or a value array) shorter than the key array before any launch, and the
    table is left untouched."""
    from paper_1908_05936_gb300.table import Table
    t = Table(O.MAP_U64_U64, 1000)
    try:
        k = to_device(np.arange(1, 101, dtype=np.uint64))
        v = to_device(np.arange(1, 101, dtype=np.uint64))
        short8 = torch.empty(99, dtype=torch.int64, device="cuda")
        short1 = torch.empty(99, dtype=torch.uint8, device="cuda")
        with pytest.raises(ValueError):
            t.insert(k, v, status=short1)
        with pytest.raises(ValueError):
            t.insert(k, short8)
        with pytest.raises(ValueError):
            t.find(k, found=short1)
        with pytest.raises(ValueError):
            t.find(k, vals_out=short8)
        with pytest.raises(ValueError):
            t.erase(k, status=short1)
        with pytest.raises(ValueError):
            t.insert_ordered(k, v, status=short1)
        with pytest.raises(ValueError):
            t.apply_mixed(torch.zeros(100, dtype=torch.uint8, device="cuda"), k, v, vals_out=short8)
        with pytest.raises(ValueError):
            t.select(keys_out=short8, cap=100)
        with pytest.raises(ValueError):
            t.find_host(np.arange(100, dtype=np.uint64), found=np.empty(99, np.uint8))
        assert t.size() == 0
        t.insert(k, v)
        f, vo = t.find(k)
        assert to_numpy(f, np.uint8).all() and np.array_equal(to_numpy(vo, np.uint64), np.arange(1, 101))
    finally:
        t.close()
