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
