"""RGB-D voxel-block stream (map<int64 packed block, int32>): per frame, find
the candidate blocks, then insert the missing ones (hc_find +
hc_insert_if_absent), against the oracle's sequential find-then-insert, with
the paper's spatial hash and with the default hash, eagerly and replayed from
a captured CUDA graph."""
from dataclasses import replace

import numpy as np
import pytest
import torch

import compare as C
from oracle import oracle as O
from paper_1908_05936_gb300 import _lib as L
from paper_1908_05936_gb300.table import Table, to_device, to_numpy
from workloads import rgbd

pytestmark = pytest.mark.gpu

PARAMS = replace(rgbd.RGBDParams(), frames=10, per_frame=40_000)


def oracle_frame(o, keys, vals):
    """find, then insert the keys the find did not see (sequential)."""
    found, _ = o.find(keys)
    status = np.full(len(keys), C.EXISTS, np.uint8)
    miss = np.nonzero(found == 0)[0]
    status[miss] = o.insert(keys[miss], vals[miss])
    return found, status


@pytest.mark.parametrize("hash_mode", [L.HASH_TESCHNER, L.HASH_MIX64])
@pytest.mark.parametrize("graph", [False, True])
def test_rgbd_stream_against_oracle(hash_mode, graph):
    from paper_1908_05936_gb300 import build
    build.build()
    frames = [rgbd.frame_keys(PARAMS, f) for f in range(PARAMS.frames)]
    vals = [rgbd.values_of(k) for k in frames]
    cap = 1 << 20
    t = Table(L.MAP_I64_I32, cap, bucket_bytes=64, hash_mode=hash_mode)
    o = O.OracleTable(O.MAP_I64_I32, cap)
    d_keys = [to_device(k) for k in frames]
    d_vals = [to_device(v) for v in vals]
    found = [torch.empty(len(k), dtype=torch.uint8, device="cuda") for k in frames]
    status = [torch.empty(len(k), dtype=torch.uint8, device="cuda") for k in frames]

    def run_frames():
        for f in range(PARAMS.frames):
            t.find(d_keys[f], found=found[f], vals_out=False)
            t.insert_if_absent(d_keys[f], d_vals[f], found[f], status=status[f])

    if graph:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            run_frames()
        t.clear()          # capture does not execute; start from empty
        torch.cuda.synchronize()
        g.replay()
    else:
        run_frames()
    torch.cuda.synchronize()
    present = []
    for f in range(PARAMS.frames):
        of, ost = oracle_frame(o, frames[f], vals[f])
        C.assert_find(to_numpy(found[f], np.uint8), None, of, None, f"frame {f} find")
        C.assert_status(frames[f], to_numpy(status[f], np.uint8), ost, f"frame {f} insert")
        present.append(of.mean())
    assert t.size() == o.size()
    gk, gv = t.dump_numpy()
    ok, ov = o.dump()
    C.assert_contents(gk, gv, ok, ov)
    assert np.mean(present[3:]) > 0.25          # candidates repeat once the camera has seen a region
    t.close()
    o.close()


@pytest.fixture(scope="module")
def full_stream():
    """The whole stream the bench times (300 frames x 400,000 candidates) and
    the oracle's per-frame find-then-insert over it."""
    p = rgbd.RGBDParams()
    frames = rgbd.all_frame_keys(p, workers=16)
    vals = [rgbd.values_of(k) for k in frames]
    o = O.OracleTable(O.MAP_I64_I32, FULL_SLOTS)
    found, status = [], []
    for f in range(p.frames):
        of, ost = oracle_frame(o, frames[f], vals[f])
        found.append(of)
        status.append(ost)
    ok, ov = o.dump()
    size = o.size()
    o.close()
    return p, frames, vals, found, status, ok, ov, size


FULL_SLOTS = 12_500_000


@pytest.mark.slow
@pytest.mark.parametrize("hash_mode", [L.HASH_TESCHNER, L.HASH_MIX64])
def test_rgbd_full_stream_against_oracle(full_stream, hash_mode):
    """The full stream in the bench's configuration (12.5 M slots, 128-byte
    buckets, the whole stream captured in one CUDA graph and replayed),
    frame by frame against the oracle: found flags, insert statuses, and the
    final contents (about 10 M blocks at load factor 0.8)."""
    from paper_1908_05936_gb300 import build
    build.build()
    p, frames, vals, ofound, ostatus, ok, ov, osize = full_stream
    t = Table(L.MAP_I64_I32, FULL_SLOTS, bucket_bytes=128, hash_mode=hash_mode)
    d_keys = [to_device(k) for k in frames]
    d_vals = [to_device(v) for v in vals]
    found = [torch.empty(len(k), dtype=torch.uint8, device="cuda") for k in frames]
    status = [torch.empty(len(k), dtype=torch.uint8, device="cuda") for k in frames]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for f in range(p.frames):
            t.find(d_keys[f], found=found[f], vals_out=False)
            t.insert_if_absent(d_keys[f], d_vals[f], found[f], status=status[f])
    t.clear()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    for f in range(p.frames):
        C.assert_find(to_numpy(found[f], np.uint8), None, ofound[f], None, f"frame {f} find")
        C.assert_status(frames[f], to_numpy(status[f], np.uint8), ostatus[f], f"frame {f} insert")
    assert t.size() == osize
    gk, gv = t.dump_numpy()
    C.assert_contents(gk, gv, ok, ov)
    assert 9_000_000 < osize < FULL_SLOTS          # about 10 M blocks, load factor about 0.8
    present = np.mean([x.mean() for x in ofound[1:]])
    assert 0.8 < present < 0.95                    # about 90 % of a frame's candidates already stored
    t.close()
