"""Served form: a continuous-batching request loop over resident tables.

Requests (insert / find / erase of a host key array on one table) arrive
over time.  The loop itself is native (`hc_server_run` in libhc.so, on the
calling host thread):

1. **Queueing.**  An arrived request joins its table's FIFO.  A table is pinned
   to one dispatch lane (a CUDA stream), so its requests reach the GPU in
   arrival order and see each other's effects in that order.
2. **Admission against the HBM budget.**  Each lane owns `depth` launch slots.
   A slot is a fixed device staging buffer (keys, values, results) plus pinned
   host staging; the slots and the resident tables are the whole HBM budget.
   A request is admitted when a free slot of its lane has room for it.  It
   waits otherwise; it is never dropped.
3. **Dispatch.**  A free slot takes the heads of its lane's FIFOs, one per
   table, while they fit, and runs one batched launch for all of them
   (`hc_batch_run`, merged mode) or one range call each (plain mode), then
   records an event.  A request whose tensors are all page-locked (as this
   module makes the results; pin the keys and values) runs in place: the
   kernels read and write host memory directly, with no copies.  Others are
   copied host->device (small requests packed into one copy) and back.
   Different lanes overlap on the device.
4. **Completion.**  A finished slot hands each request its results and its
   completion time (arrival to the host holding the results).

A request larger than a slot (and not page-locked) is cut into chunks that
run in order; a request
with a deadline is dropped (``rc`` = HC_ERR_TIMEOUT, nothing of it runs) if
it is still waiting for a slot when the deadline passes.  ``run`` serves a
list of requests with arrival times on the calling thread; ``start`` runs
the loop on a native thread of its own, to which ``submit`` hands requests
from any Python thread while it runs (``wait`` blocks for one, ``stop``
ends the loop).

This module only marshals requests and results; every table stays resident
in HBM throughout.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from .table import Table


@dataclass
class ServedRequest:
    """One request: `op` on table `table` over the host (pinned) int64 key
    bit patterns `keys`; `vals` are the values of a map insert."""
    rid: int
    table: int
    op: int
    keys: torch.Tensor
    vals: torch.Tensor | None
    arrival: float = 0.0                  # seconds after the start of the run (set by submit)
    status: np.ndarray | None = None      # insert/erase status, or found flags
    values: np.ndarray | None = None      # find values (maps)
    done: float = -1.0
    deadline: float = 0.0                 # seconds after arrival to be dispatched by (0: none)
    rc: int = -1                          # HC_OK, or HC_ERR_TIMEOUT when dropped at its deadline

    @property
    def n(self) -> int:
        return self.keys.numel()


class Server:
    def __init__(self, tables: list[Table], slot_bytes: int = 64 << 20, lanes: int = 4, depth: int = 2,
                 merge: bool = True, max_items: int = 256, batch_config: tuple = (0, 1, 256, 0, 0, 0)):
        self.lib = L.load()
        self.tables = tables
        self.lanes, self.depth, self.merge = lanes, depth, merge
        self.max_items = max_items if merge else 1
        self.slot_bytes = slot_bytes
        handles = (ctypes.c_void_p * len(tables))(*[t.handle for t in tables])
        cfg = L.ServeConfig(lanes, depth, slot_bytes, int(merge), max_items, L.BatchConfig(*batch_config))
        h = ctypes.c_void_p()
        L.check(self.lib.hc_server_create(ctypes.byref(h), handles, len(tables), ctypes.byref(cfg)))
        self.h = h
        self.resident_bytes = sum(t.stats()["table_bytes"] for t in tables)

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            L.check(self.lib.hc_server_destroy(self.h))
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def hbm_budget(self) -> dict:
        slots = self.lanes * self.depth
        desc = int(self.lib.hc_batch_scratch_bytes(self.max_items))
        return {"resident_tables_bytes": self.resident_bytes, "launch_slots_bytes": slots * (self.slot_bytes + desc),
                "slots": slots, "slot_bytes": self.slot_bytes}

    def run(self, requests: list[ServedRequest], realtime: bool = True, timeout_s: float = 600.0) -> dict:
        """Serve `requests` (sorted by arrival).  With realtime=False every
        request counts as arrived at time 0 (a capacity measurement)."""
        n = len(requests)
        arr = (L.Request * n)()
        # every request's results in one page-locked buffer, so that large
        # results are copied straight into place
        sizes = []
        for r in requests:
            t = self.tables[r.table]
            vb = t.val_bytes if (r.op == L.OP_FIND and t.is_map) else 0
            sizes.append((-(-r.n // 8) * 8, r.n * vb))
        out = torch.empty(max(1, sum(a + b for a, b in sizes)), dtype=torch.uint8).pin_memory().numpy()
        off = 0
        for i, r in enumerate(requests):
            t = self.tables[r.table]
            if not r.keys.is_contiguous() or r.keys.element_size() != t.key_bytes:
                raise TypeError(f"request {r.rid}: keys must be contiguous with {t.key_bytes}-byte elements")
            sb, vbytes = sizes[i]
            r.status = out[off:off + r.n]
            r.values = out[off + sb:off + sb + vbytes].view(np.int32 if t.val_bytes == 4 else np.int64) \
                if vbytes else None
            off += sb + vbytes
            arr[i] = self._c_request(r, float(r.arrival) if realtime else 0.0)
        st = L.ServeStats()
        L.check(self.lib.hc_server_run(self.h, arr, n, int(realtime), float(timeout_s), ctypes.byref(st)))
        for i, r in enumerate(requests):
            r.done = arr[i].done
            r.rc = arr[i].rc
        return self._stats(st)

    def _c_request(self, r: ServedRequest, arrival: float) -> L.Request:
        t = self.tables[r.table]
        return L.Request(r.table, r.op, r.keys.data_ptr(), r.vals.data_ptr() if (r.op == L.OP_INSERT and t.is_map)
                         else None, r.n, r.status.ctypes.data, r.values.ctypes.data if r.values is not None else None,
                         arrival, float(r.deadline), -1.0, -1, 0)

    def _stats(self, st: L.ServeStats) -> dict:
        return {"requests": st.requests, "ops": st.ops, "wall_s": round(st.wall_s, 4),
                "mops": round(st.ops / st.wall_s / 1e6, 2) if st.wall_s > 0 else 0.0, "launches": st.launches,
                "p50_ms": round(st.p50_ms, 3), "p99_ms": round(st.p99_ms, 3), "p999_ms": round(st.p999_ms, 3),
                "max_ms": round(st.max_ms, 3), "queued_max": st.queued_max, "timed_out": st.timed_out,
                "merge": self.merge, "lanes": self.lanes, "depth": self.depth}

    # ---- the loop on its own thread, fed while it runs -------------------

    def start(self):
        """Start the native loop on a thread of its own (hc_server_start)."""
        L.check(self.lib.hc_server_start(self.h))

    def submit(self, r: ServedRequest):
        """Hand `r` to the running loop; callable from any thread.  Its
        result arrays are allocated here (page-locked); read them after
        wait(r)."""
        t = self.tables[r.table]
        if not r.keys.is_contiguous() or r.keys.element_size() != t.key_bytes:
            raise TypeError(f"request {r.rid}: keys must be contiguous with {t.key_bytes}-byte elements")
        vb = t.val_bytes if (r.op == L.OP_FIND and t.is_map) else 0
        sb = -(-r.n // 8) * 8
        out = torch.empty(max(1, sb + r.n * vb), dtype=torch.uint8).pin_memory().numpy()
        r.status = out[:r.n]
        r.values = out[sb:sb + r.n * vb].view(np.int32 if t.val_bytes == 4 else np.int64) if vb else None
        r._out = out                                   # keeps the buffer (and its tensor) alive
        r._c = self._c_request(r, 0.0)
        L.check(self.lib.hc_server_submit(self.h, ctypes.byref(r._c)))

    def wait(self, r: ServedRequest, timeout_s: float = 60.0) -> int:
        """Block until `r` is done; returns HC_OK, or HC_ERR_TIMEOUT when it
        was dropped at its deadline (other errors raise)."""
        rc = self.lib.hc_server_wait(self.h, ctypes.byref(r._c), float(timeout_s))
        r.arrival, r.done, r.rc = r._c.arrival, r._c.done, r._c.rc
        if rc != L.ERR_TIMEOUT or r.rc != L.ERR_TIMEOUT:
            L.check(rc)
        return rc

    def stop(self) -> dict:
        """Serve what was submitted, end the loop, return its statistics."""
        st = L.ServeStats()
        L.check(self.lib.hc_server_stop(self.h, ctypes.byref(st)))
        return self._stats(st)
