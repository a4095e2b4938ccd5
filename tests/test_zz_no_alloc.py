"""hc_batch_run_noalloc: the batched form for callers that may not allocate
device memory (a process whose GPU memory belongs to another allocator's
pool, or a latency-bound request loop that cannot afford the device-wide
synchronisation a cudaMalloc brings).  It must give the same results as a
batch built with hc_batch_create and launched, on two calls in a row, with
the tables, keys and outputs all supplied by the caller.

This file is collected last on purpose, so that a run that stops at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import compare as C
from paper_1908_05936_gb300 import _lib as L
from paper_1908_05936_gb300.batch import Batch, Item
from paper_1908_05936_gb300.table import Table, to_device, to_numpy
from workloads import recipes

pytestmark = pytest.mark.gpu


def _setup(seed):
    """Two identical sets of tables and per-item output buffers."""
    from paper_1908_05936_gb300 import build
    build.build()
    slots = recipes.multi_table_slots(24, 10, 15, seed=seed)
    ops = [recipes.multi_table_ops(int(s), t, seed=seed) for t, s in enumerate(slots)]
    sides = []
    for _ in range(2):
        tables, items, outs = [], [], []
        for t, (s, o) in enumerate(zip(slots, ops)):
            kind = L.SET_U64 if t % 2 == 0 else L.MAP_U64_U64
            tab = Table(kind, int(s), bucket_bytes=(32, 64, 128)[t % 3])
            ki, kf, ke = to_device(o.insert_keys), to_device(o.find_keys), to_device(o.erase_keys)
            vi = to_device(o.insert_keys ^ np.uint64(0x5bd1e995)) if kind == L.MAP_U64_U64 else None
            si = torch.empty(len(o.insert_keys), dtype=torch.uint8, device="cuda")
            ff = torch.empty(len(o.find_keys), dtype=torch.uint8, device="cuda")
            fv = torch.empty(len(o.find_keys), dtype=torch.int64, device="cuda") if kind == L.MAP_U64_U64 else None
            se = torch.empty(len(o.erase_keys), dtype=torch.uint8, device="cuda")
            items += [Item(tab, L.OP_INSERT, ki, vi, si), Item(tab, L.OP_FIND, kf, None, ff, fv),
                      Item(tab, L.OP_ERASE, ke, None, se)]
            tables.append(tab)
            outs.append((si, ff, fv, se))
        sides.append((tables, items, outs))
    return ops, sides


def _item_array(items):
    arr = (L.BatchItem * len(items))()
    for i, it in enumerate(items):
        arr[i] = L.BatchItem(it.table.handle, it.op, 0, it.keys.data_ptr(),
                             it.vals.data_ptr() if it.vals is not None else None, it.keys.numel(),
                             it.out.data_ptr() if it.out is not None else None,
                             it.vals_out.data_ptr() if it.vals_out is not None else None)
    return arr


@pytest.mark.parametrize("kpt,block", [(1, 256), (4, 128)], ids=["lock-step", "streaming"])
def test_noalloc_matches_batch_on_two_calls(kpt, block):
    """Same shape on both entry points: the lock-step phases, and the
    streaming phases with their dynamic shared memory."""
    ops, ((tab_a, items_a, outs_a), (tab_b, items_b, outs_b)) = _setup(seed=7)
    lib = L.load()
    batch = Batch(items_a, lane_bytes=0, keys_per_group=kpt, block=block, tile=1024,
                  use_graph=False)                   # the existing entry point
    arr_b = _item_array(items_b)
    cfg = L.BatchConfig(0, kpt, block, 0, 1024, 0)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        batch.launch()
        L.check(lib.hc_batch_run_noalloc(arr_b, len(items_b), ctypes.byref(cfg), stream))
        torch.cuda.synchronize()
        for t, o in enumerate(ops):
            sa, fa, va, ea = outs_a[t]
            sb, fb, vb, eb = outs_b[t]
            C.assert_status(o.insert_keys, to_numpy(sb, np.uint8), to_numpy(sa, np.uint8), f"call {call} table {t} insert")
            C.assert_find(to_numpy(fb, np.uint8), to_numpy(vb, np.uint64) if vb is not None else None,
                          to_numpy(fa, np.uint8), to_numpy(va, np.uint64) if va is not None else None,
                          f"call {call} table {t} find")
            C.assert_status(o.erase_keys, to_numpy(eb, np.uint8), to_numpy(ea, np.uint8), f"call {call} table {t} erase")
            ka, vka = tab_a[t].dump_numpy()
            kb, vkb = tab_b[t].dump_numpy()
            C.assert_contents(kb, vkb, ka, vka, f"call {call} table {t} contents")
    batch.close()
    for tb in tab_a + tab_b:
        tb.close()


def test_noalloc_rejects_too_many_items():
    from paper_1908_05936_gb300 import build
    build.build()
    lib = L.load()
    t = Table(L.SET_U64, 64)
    keys = torch.zeros(1, dtype=torch.int64, device="cuda")
    found = torch.zeros(1, dtype=torch.uint8, device="cuda")
    arr = (L.BatchItem * 1025)()
    for i in range(1025):
        arr[i] = L.BatchItem(t.handle, L.OP_FIND, 0, keys.data_ptr(), None, 1, found.data_ptr(), None)
    rc = lib.hc_batch_run_noalloc(arr, 1025, None, None)
    assert rc == L.ERR_ARG
    assert b"1024" in lib.hc_last_error()
    t.close()
