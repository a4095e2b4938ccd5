"""short3 block keys (Section 4.1's voxel-block map keyed by three signed
16-bit coordinates): packing on the device against the packing computed here,
a map<int64,int32> with the spatial hash on short3 against the oracle and
against the same calls on a mix64 table, the short3 box selection against the
oracle, and the in-kernel functions on such a table."""
import numpy as np
import pytest
import torch

import compare as C
from gpu_pair import Pair, value_for
from oracle import oracle as O
from paper_1908_05936_gb300 import _lib as L
from paper_1908_05936_gb300 import device_api as D
from paper_1908_05936_gb300.table import Table, pack_short3, to_device, to_numpy, unpack_short3

pytestmark = pytest.mark.gpu


def _coords(n, rng, spread=40):
    c = rng.integers(-spread, spread, size=(n, 3)).astype(np.int16)
    edge = np.array([[-32768, 32767, 0], [32767, -32768, -1], [-1, -1, -1], [0, 0, 0]], dtype=np.int16)
    return np.concatenate([c, edge])


def _pack_here(c):
    u = c.astype(np.int64) & 0xFFFF
    return (u[:, 0] | (u[:, 1] << 16) | (u[:, 2] << 32)).astype(np.int64)


def test_pack_unpack_bits():
    rng = np.random.default_rng(1300)
    c = np.concatenate([rng.integers(-32768, 32768, size=(100000, 3)).astype(np.int16), _coords(0, rng)])
    keys = pack_short3(torch.from_numpy(c).cuda())
    assert np.array_equal(to_numpy(keys, np.int64), _pack_here(c))
    back = unpack_short3(keys).cpu().numpy()
    assert np.array_equal(back, c)
    assert pack_short3(torch.empty((0, 3), dtype=torch.int16, device="cuda")).numel() == 0


@pytest.mark.parametrize("bb", (32, 64, 128))
def test_short3_map_matches_oracle_and_mix64(bb):
    rng = np.random.default_rng(1310 + bb)
    p = Pair(O.MAP_I64_I32, 30000, bucket_bytes=bb, hash_mode=L.HASH_TESCHNER_SHORT3)
    q = Pair(O.MAP_I64_I32, 30000, bucket_bytes=bb, hash_mode=L.HASH_MIX64)
    try:
        dom = np.unique(_pack_here(_coords(20000, rng)))
        for b, n in enumerate((1, 1000, 15000, 15000)):
            keys = dom[rng.integers(0, len(dom), size=n)]
            vals = value_for(O.MAP_I64_I32, keys, salt=b)
            g1, _ = p.insert(keys, vals)
            g2, _ = q.insert(keys, vals)
            query = np.concatenate([keys, dom[rng.integers(0, len(dom), size=n)]])
            f1, v1 = p.find(query)
            f2, v2 = q.find(query)
            assert np.array_equal(f1, f2) and np.array_equal(v1, v2)
            p.erase(keys[::3])
            q.erase(keys[::3])
        p.check()
        q.check()
        for box in ((-10, 10, -40, 0, -5, 39), (-32768, 0, -32768, 32767, -1, -1)):
            ko, vo, cnt = p.g.select(L.PRED_SHORT3_BOX, box=box)
            n = int(cnt.item())
            gk, gv = to_numpy(ko[:n], np.int64), to_numpy(vo[:n], np.int32)
            ok, ov = p.o.select(O.PRED_SHORT3_BOX, box=box)
            order = np.argsort(C.bits(gk), kind="stable")
            C.assert_contents(gk[order], gv[order], ok, ov, "short3 box selection")
    finally:
        p.close()
        q.close()


def test_in_kernel_functions_on_short3_map():
    rng = np.random.default_rng(1320)
    p = Pair(O.MAP_I64_I32, 20000, bucket_bytes=32, hash_mode=L.HASH_TESCHNER_SHORT3)
    try:
        keys = np.unique(_pack_here(_coords(8000, rng)))
        vals = value_for(O.MAP_I64_I32, keys)
        st, _, _ = D.apply(p.g, to_device(keys), L.OP_INSERT, vals=to_device(vals))
        C.assert_status(keys, to_numpy(st, np.uint8), p.o.insert(keys, vals), "in-kernel insert")
        query = np.concatenate([keys, _pack_here(_coords(3000, rng))])
        f, vo, _ = D.apply(p.g, to_device(query), L.OP_FIND, vals_out=True)
        of, ov = p.o.find(query)
        C.assert_find(to_numpy(f, np.uint8), to_numpy(vo, np.int32), of, ov)
        p.check()
    finally:
        p.close()


def test_mixed_and_pack_empty_calls():
    """n = 0 is a no-op for the mixed batch and the short3 conversions."""
    t = Table(O.SET_U64, 100)
    try:
        e = torch.empty(0, dtype=torch.int64, device="cuda")
        st, _ = t.apply_mixed(torch.empty(0, dtype=torch.uint8, device="cuda"), e)
        assert st.numel() == 0
        assert unpack_short3(e).shape == (0, 3)
        assert t.size() == 0
    finally:
        t.close()
