"""The in-kernel function form (include/hc_device.cuh, Section 4.1) driven
through the user kernels of libhc_examples.so:
  - one kind of operation per launch against the oracle (statuses as a
    multiset per key, find results exactly, contents and size), mixed with
    range calls on the same table;
  - positions: every call on one key reports one position, distinct keys
    distinct positions, find agrees with insert;
  - overflow: in-kernel inserts claim EMPTY slots only, so tombstones are not
    reused until rehash (invariants, the overflowing subset is not fixed);
  - free-running mixed insert / find / erase on one table in one launch:
    for every key some serial order of its operations gives the recorded
    results (Section 4, "Guarantees"), no key is stored twice, map values
    are never seen torn;
  - Section 4.1's update-set kernel against the oracle."""
import numpy as np
import pytest
import torch

import compare as C
import linearizable as LZ
from gpu_pair import CLAIM_PATTERN, RESERVED, Pair, edge_keys, random_keys, value_for
from oracle import oracle as O
from paper_1908_05936_gb300 import _lib as L
from paper_1908_05936_gb300 import device_api as D
from paper_1908_05936_gb300.table import Table, to_device, to_numpy

pytestmark = pytest.mark.gpu

KINDS = (O.SET_U32, O.SET_U64, O.MAP_I64_I32, O.MAP_U64_U64)


def _vals_dev(p, keys, salt=0):
    v = value_for(p.kind, keys, salt)
    return to_device(v) if v is not None else None


def dev_insert(p, keys, salt=0, check=True):
    st, _, pos = D.apply(p.g, to_device(keys), L.OP_INSERT, vals=_vals_dev(p, keys, salt), pos_out=True)
    gs = to_numpy(st, np.uint8)
    os_ = p.o.insert(keys, value_for(p.kind, keys, salt))
    if check:
        C.assert_status(keys, gs, os_, "in-kernel insert status")
    return gs, to_numpy(pos, np.int64)


def dev_find(p, keys):
    st, vo, pos = D.apply(p.g, to_device(keys), L.OP_FIND, vals_out=p.is_map, pos_out=True)
    gf = to_numpy(st, np.uint8)
    gv = to_numpy(vo, O.VAL_DTYPE[p.kind]) if p.is_map else None
    of, ov = p.o.find(keys)
    C.assert_find(gf, gv, of, ov, "in-kernel find")
    return gf, to_numpy(pos, np.int64)


def dev_erase(p, keys):
    st, _, _ = D.apply(p.g, to_device(keys), L.OP_ERASE)
    gs = to_numpy(st, np.uint8)
    C.assert_status(keys, gs, p.o.erase(keys), "in-kernel erase status")
    return gs


def _positions_consistent(keys, pos, ok):
    """Equal keys share one position; distinct keys have distinct positions."""
    kb = C.bits(keys)[ok]
    ps = pos[ok]
    seen = {}
    for k, q in zip(kb.tolist(), ps.tolist()):
        assert q >= 0
        assert seen.setdefault(k, q) == q, "one key at two positions"
    assert len(set(seen.values())) == len(seen), "two keys at one position"
    return seen


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bb", (32, 64, 128))
def test_in_kernel_ops_match_oracle(kind, bb):
    rng = np.random.default_rng(500 + kind * 7 + bb)
    p = Pair(kind, 60000, bucket_bytes=bb)
    dom = np.concatenate([random_keys(kind, 12000, rng), edge_keys(kind)])
    try:
        for b, n in enumerate((0, 1, 100, 5000, 12000)):
            keys = dom[rng.integers(0, len(dom), size=n)]
            st, pos = dev_insert(p, keys, salt=b)
            where = _positions_consistent(keys, pos, st <= 1)
            q = np.concatenate([keys, random_keys(kind, n, rng)])
            f, fpos = dev_find(p, q)
            for k, fp in zip(C.bits(q)[f == 1].tolist(), fpos[f == 1].tolist()):
                if k in where:
                    assert where[k] == fp, "find and insert disagree on the position"
            assert (fpos[f == 0] == -1).all()
            dev_erase(p, keys[::3])
            p.check()
        # range calls and in-kernel calls on one table
        extra = random_keys(kind, 3000, rng)
        p.insert(extra, value_for(kind, extra, salt=9))
        dev_find(p, np.concatenate([extra, dom[:2000]]))
        p.find(dom)
        dev_erase(p, extra[::2])
        p.erase(dom[::5])
        p.check()
        # a rehash moves the slots: a fresh view still finds everything
        p.rehash(40000)
        dev_find(p, dom)
        st, _ = dev_insert(p, random_keys(kind, 1000, rng), salt=11)
        p.check()
    finally:
        p.close()


@pytest.mark.parametrize("kind", KINDS)
def test_in_kernel_overflow_and_no_tombstone_reuse(kind):
    rng = np.random.default_rng(600 + kind)
    t = Table(kind, 100, bucket_bytes=32)
    reserved = {int(x) for x in C.bits(np.array(RESERVED[kind]))}
    try:
        keys = random_keys(kind, 300, rng)
        keys = keys[[int(x) not in reserved for x in C.bits(keys)]]
        vals = value_for(kind, keys)
        st, _, pos = D.apply(t, to_device(keys), L.OP_INSERT, vals=to_device(vals) if vals is not None else None,
                             pos_out=True)
        st = to_numpy(st, np.uint8)
        gk, _ = t.dump_numpy()
        stored = {int(x) for x in C.bits(gk)}
        C.check_overflow_insert(keys, st, set(), 100, stored, set())
        assert (to_numpy(pos, np.int64)[st == C.OVERFLOW] == -1).all()
        assert t.status() == L.ERR_OVERFLOW
        # erase half: tombstones; in-kernel inserts do not reuse them
        inserted = keys[st == C.INSERTED]
        es = to_numpy(D.apply(t, to_device(inserted[:50]), L.OP_ERASE)[0], np.uint8)
        assert (es == C.ERASED).all()
        s = t.stats()
        assert (s["live"], s["used"]) == (50, 100)
        fresh = random_keys(kind, 60, rng)
        fresh = fresh[[int(x) not in reserved and int(x) not in stored for x in C.bits(fresh)]]
        fv = value_for(kind, fresh)
        fst = to_numpy(D.apply(t, to_device(fresh), L.OP_INSERT,
                               vals=to_device(fv) if fv is not None else None)[0], np.uint8)
        assert (fst == C.OVERFLOW).all()
        assert t.size() == 50
        # rehash purges the tombstones: the same keys now fit
        t.rehash(100)
        fst = to_numpy(D.apply(t, to_device(fresh[:50]), L.OP_INSERT,
                               vals=to_device(fv[:50]) if fv is not None else None)[0], np.uint8)
        assert (fst == C.INSERTED).all()
        assert t.size() == 100
    finally:
        t.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bb", (32, 128))
def test_in_kernel_inserts_reuse_slots_after_clear_and_rehash(kind, bb):
    """In-kernel inserts claim EMPTY slots only; hc_clear makes every slot
    EMPTY again and hc_rehash moves the keys to new slots (for maps with new
    lock bits, allocated by the rehash).  Fill to a load factor of 0.85
    in-kernel, erase some, clear, fill again with keys that overlap the first
    set, rehash, fill on: every status, the contents and the size against
    the oracle, and no retry bound is reached."""
    rng = np.random.default_rng(700 + kind + bb)
    reserved = {int(x) for x in C.bits(np.array(RESERVED[kind]))}
    p = Pair(kind, 4096, bucket_bytes=bb)
    try:
        def fresh(n):
            k = random_keys(kind, n, rng)
            return k[[int(x) not in reserved for x in C.bits(k)]]
        first = fresh(3480)
        dev_insert(p, first)
        dev_erase(p, first[:500])
        p.check()
        p.clear()
        second = np.concatenate([first[1000:2500], fresh(1980)])
        st, _ = dev_insert(p, second, salt=1)
        assert (st != C.OVERFLOW).all()
        p.check()
        assert p.g.status() == L.OK
        assert p.rehash(8192)
        dev_insert(p, np.concatenate([second[:1000], fresh(2500)]), salt=2)
        p.check()
        assert p.g.status() == L.OK
    finally:
        p.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bb", (32, 128))
def test_free_running_mixed_ops(kind, bb):
    """Inserts, finds and erases of a small key domain from 2^18 threads in
    one launch (about 64 operations per key)."""
    rng = np.random.default_rng(700 + kind * 3 + bb)
    t = Table(kind, 1 << 19, bucket_bytes=bb)
    dom = np.concatenate([random_keys(kind, 1 << 12, rng), edge_keys(kind)])
    dom = dom[np.unique(C.bits(dom), return_index=True)[1]]
    try:
        pre = dom[rng.random(len(dom)) < 0.5]
        pv = value_for(kind, pre)
        t.insert(to_device(pre), to_device(pv) if pv is not None else None)
        before = {int(x) for x in C.bits(pre)}
        for rep in range(3):
            n = 1 << 18
            keys = dom[rng.integers(0, len(dom), size=n)]
            ops = rng.choice(np.array([0, 1, 2], dtype=np.uint8), size=n, p=[0.4, 0.3, 0.3])
            vals = value_for(kind, keys)
            st, vo, pos = D.apply(t, to_device(keys), to_device(ops), vals=to_device(vals) if vals is not None else None,
                                  vals_out=t.is_map, pos_out=True)
            st = to_numpy(st, np.uint8)
            gk, gv = t.dump_numpy()
            kb = C.bits(gk)
            assert len(np.unique(kb)) == len(kb), "a key stored twice"
            assert t.size() == len(kb)
            after = {int(x) for x in kb}
            assert LZ.check_history(C.bits(keys), ops, st, before, after) == []
            untouched = {int(x) for x in C.bits(dom)} - {int(x) for x in C.bits(keys)}
            assert {k for k in untouched if k in before} == {k for k in untouched if k in after}
            if t.is_map:
                got = to_numpy(vo, O.VAL_DTYPE[kind])
                found = (ops == 1) & (st == 1)
                assert np.array_equal(C.bits(got[found]), C.bits(vals[found])), "a find saw a value not stored"
                assert np.array_equal(C.bits(gv), C.bits(value_for(kind, gk)))
            assert t.status() == L.OK
            before = after
    finally:
        t.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bb", (32, 64, 128))
def test_apply_mixed_serial_order_per_key(kind, bb):
    """hc_apply_mixed (the library's free-running mixed batch) under the same
    per-key check, with 2^20 operations over 2^14 keys."""
    rng = np.random.default_rng(750 + kind + bb)
    t = Table(kind, 1 << 21, bucket_bytes=bb)
    dom = np.concatenate([random_keys(kind, 1 << 14, rng), edge_keys(kind)])
    dom = dom[np.unique(C.bits(dom), return_index=True)[1]]
    try:
        before = set()
        for rep in range(2):
            n = 1 << 20
            keys = dom[rng.integers(0, len(dom), size=n)]
            ops = rng.choice(np.array([0, 1, 2], dtype=np.uint8), size=n, p=[0.5, 0.25, 0.25])
            vals = value_for(kind, keys)
            st, vo = t.apply_mixed(to_device(ops), to_device(keys), to_device(vals) if vals is not None else None,
                                   vals_out=t.is_map)
            st = to_numpy(st, np.uint8)
            gk, gv = t.dump_numpy()
            kb = C.bits(gk)
            assert len(np.unique(kb)) == len(kb) == t.size()
            after = {int(x) for x in kb}
            assert LZ.check_history(C.bits(keys), ops, st, before, after) == []
            if t.is_map:
                got = to_numpy(vo, O.VAL_DTYPE[kind])
                found = (ops == 1) & (st == 1)
                assert np.array_equal(C.bits(got[found]), C.bits(vals[found]))
                assert not C.bits(got[~found]).any(), "a value out where no key was found"
                assert np.array_equal(C.bits(gv), C.bits(value_for(kind, gk)))
            assert t.status() == L.OK
            before = after
    finally:
        t.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bb", (32, 128))
def test_apply_mixed_on_a_table_that_fills_up(kind, bb):
    """hc_apply_mixed on a 96-slot table: 2^14 mixed operations (60 / 20 / 20
    insert / find / erase) over 400 keys plus the edge patterns, so the
    table runs out of EMPTY slots during the launch (inserts do not reuse
    tombstones).  Every insert reports INSERTED, EXISTS or OVERFLOW; per key
    the results admit a serial order in which an OVERFLOW insert found the
    key absent; no key is stored twice; at most the capacity is stored in
    slots; found values are the inserted ones."""
    rng = np.random.default_rng(820 + kind + bb)
    cap = 96
    t = Table(kind, cap, bucket_bytes=bb)
    dom = np.concatenate([random_keys(kind, 400, rng), edge_keys(kind)])
    dom = dom[np.unique(C.bits(dom), return_index=True)[1]]
    side = {int(x) for x in C.bits(np.array(RESERVED[kind]))}
    try:
        pre = dom[rng.random(len(dom)) < 0.1]
        pv = value_for(kind, pre)
        t.insert(to_device(pre), to_device(pv) if pv is not None else None)
        before = {int(x) for x in C.bits(t.dump_numpy()[0])}
        for rep in range(2):
            n = 1 << 14
            keys = dom[rng.integers(0, len(dom), size=n)]
            ops = rng.choice(np.array([0, 1, 2], dtype=np.uint8), size=n, p=[0.6, 0.2, 0.2])
            vals = value_for(kind, keys)
            st, vo = t.apply_mixed(to_device(ops), to_device(keys), to_device(vals) if vals is not None else None,
                                   vals_out=t.is_map)
            st = to_numpy(st, np.uint8)
            gk, gv = t.dump_numpy()
            kb = C.bits(gk)
            assert len(np.unique(kb)) == len(kb) == t.size(), "a key stored twice, or size off"
            assert sum(1 for x in kb.tolist() if int(x) not in side) <= cap
            after = {int(x) for x in kb}
            assert LZ.check_history(C.bits(keys), ops, st, before, after, overflow=True) == []
            if t.is_map:
                got = to_numpy(vo, O.VAL_DTYPE[kind])
                found = (ops == 1) & (st == 1)
                assert np.array_equal(C.bits(got[found]), C.bits(vals[found]))
                assert np.array_equal(C.bits(gv), C.bits(value_for(kind, gk)))
            assert t.status() in (L.OK, L.ERR_OVERFLOW)
            before = after
        assert (st == C.OVERFLOW).any(), "the table never filled up"
    finally:
        t.close()


@pytest.mark.parametrize("kind", [O.MAP_I64_I32, O.MAP_U64_U64])
@pytest.mark.parametrize("how", ["range", "in-kernel"])
def test_in_kernel_map_inserts_past_a_stored_claim_pattern_key(kind, how):
    """A map insert in a kernel waits only for claims in progress, never for
    the stored key whose bit pattern equals the claim marker.  That key is put
    into a 64-slot table (by a range call or in-kernel), most of the table is
    filled around it in-kernel, so that nearly every later probe crosses its
    bucket, then it is erased and inserted again while other keys go in: every
    status, value and the contents against the oracle, and no retry bound
    reached (a wait on the stored key would end at that bound).  In-kernel
    inserts do not reuse tombstones, so the script stays below the capacity
    (at most 59 of 64 slots used before the rehash)."""
    rng = np.random.default_rng(900 + kind)
    claim = np.array([CLAIM_PATTERN[kind]])
    p = Pair(kind, 64, bucket_bytes=32)
    try:
        if how == "range":
            p.insert(claim, value_for(kind, claim))
        else:
            dev_insert(p, claim)
        for rep in range(3):
            keys = np.concatenate([random_keys(kind, 15, rng), claim])
            dev_insert(p, keys, salt=rep)
            p.check()
            assert p.g.status() == L.OK
            dev_find(p, np.concatenate([keys, claim]))
        dev_erase(p, claim)
        p.check()
        keys = np.concatenate([claim, random_keys(kind, 6, rng), claim])
        dev_insert(p, keys, salt=7)
        p.check()
        p.erase(claim)
        dev_find(p, claim)
        p.insert(claim, value_for(kind, claim, salt=8))
        dev_insert(p, np.concatenate([claim, random_keys(kind, 4, rng)]), salt=9)
        p.check()
        assert p.rehash(64)
        dev_find(p, claim)
        dev_erase(p, claim)
        p.check()
        assert p.g.status() == L.OK
    finally:
        p.close()


def _pack21(x, y, z):
    m = np.int64(0x1FFFFF)
    return ((x & m) | ((y & m) << 21) | ((z & m) << 42)).astype(np.int64)


def test_update_set_example():
    """Section 4.1's compute-update-set kernel: every block and each of its 7
    neighbours towards -x, -y, -z that the block map contains goes into the
    update set.  Expected set from the oracle's map."""
    rng = np.random.default_rng(800)
    c = np.stack(np.meshgrid(*[np.arange(-20, 20)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.int64)
    c = c[rng.random(len(c)) < 0.3]
    keys = _pack21(c[:, 0], c[:, 1], c[:, 2])
    m = Table(O.MAP_I64_I32, 40000, bucket_bytes=32, hash_mode=L.HASH_TESCHNER)
    s = Table(O.SET_U64, 100000, bucket_bytes=32)
    om = O.OracleTable(O.MAP_I64_I32, 40000)
    try:
        vals = value_for(O.MAP_I64_I32, keys)
        m.insert(to_device(keys), to_device(vals))
        om.insert(keys, vals)
        q = rng.integers(-21, 21, size=(6000, 3)).astype(np.int64)
        blocks = _pack21(q[:, 0], q[:, 1], q[:, 2])
        D.update_set(m, s, to_device(blocks))
        cand = np.concatenate([_pack21(q[:, 0] - (j & 1), q[:, 1] - ((j >> 1) & 1), q[:, 2] - ((j >> 2) & 1))
                               for j in range(8)])
        present, _ = om.find(cand)
        expected = np.unique(cand[present == 1].view(np.uint64))
        gk, _ = s.dump_numpy()
        assert np.array_equal(np.sort(gk.view(np.uint64)), expected)
        assert s.size() == len(expected)
    finally:
        m.close()
        s.close()
        om.close()
