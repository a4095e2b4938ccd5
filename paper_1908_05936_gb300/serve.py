"""Served form: a continuous-batching request loop over resident tables.

Requests (insert / find / erase of a key array on one table) arrive over time.
The loop runs these steps, in order, until every request has completed:

1. **Queueing.**  An arrived request joins its table's FIFO.  A table is pinned
   to one dispatch lane (a CUDA stream), so its requests reach the GPU in
   arrival order and see each other's effects in that order.
2. **Admission against the HBM budget.**  Each lane owns `depth` launch slots.
   A slot is a fixed device staging buffer (keys, values, results) plus pinned
   host staging; the slots and the resident tables are the whole HBM budget.
   A request is admitted when a free slot of its lane has room for it.  It
   waits otherwise; it is never dropped.
3. **Dispatch.**  A free slot takes the heads of its lane's FIFOs, one per
   table, while they fit.  The heads of different tables never interact.  It
   then copies their keys host->device (small requests packed into one copy),
   runs one batched launch for all of them (`hc_batch_run`, merged mode) or
   one range call each (plain mode), copies the results device->host, and
   records an event.  Requests that arrive while other slots are on the GPU
   are admitted into the next free slot.  Different lanes overlap on the
   device.
4. **Completion.**  A finished slot hands each request its results, fixes its
   latency (arrival to the host holding the results) and becomes free again.

Every table stays resident in HBM throughout.
"""
from __future__ import annotations

import ctypes
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L
from .table import Table

PACK_LIMIT = 1 << 16        # requests up to this many keys are packed into the slot's host staging


def _round(x: int) -> int:
    return (x + 255) // 256 * 256


@dataclass
class ServedRequest:
    """One request: `op` on table `table` over the host (pinned) int64 key
    bit patterns `keys`; `vals` are the values of a map insert."""
    rid: int
    table: int
    op: int
    keys: torch.Tensor
    vals: torch.Tensor | None
    arrival: float                        # seconds after the start of the run
    status: np.ndarray | None = None      # insert/erase status, or found flags
    values: np.ndarray | None = None      # find values (maps)
    admitted: float = -1.0
    done: float = -1.0

    @property
    def n(self) -> int:
        return self.keys.numel()


@dataclass
class _Slot:
    lane: int
    d_buf: torch.Tensor          # device staging (HBM budget)
    h_in: torch.Tensor           # pinned host staging of inputs
    h_out: torch.Tensor          # pinned host staging of results
    desc: torch.Tensor           # device descriptors for hc_batch_run
    items: ctypes.Array          # host descriptors, reused by every launch of the slot
    done_event: torch.cuda.Event # reused completion event
    event: torch.cuda.Event | None = None
    reqs: list = field(default_factory=list)
    layout: list = field(default_factory=list)


class Server:
    def __init__(self, tables: list[Table], slot_bytes: int = 64 << 20, lanes: int = 4, depth: int = 2,
                 merge: bool = True, max_items: int = 256, batch_config: tuple = (0, 1, 256, 0, 1024, 0)):
        self.lib = L.load()
        self.tables = tables
        self.lanes = lanes
        self.depth = depth
        self.merge = merge
        self.max_items = max_items
        self.cfg = L.BatchConfig(*batch_config)
        self.streams = [torch.cuda.Stream() for _ in range(lanes)]
        desc_bytes = self.lib.hc_batch_scratch_bytes(max_items)
        self.slots = []
        for lane in range(lanes):
            for _ in range(depth):
                self.slots.append(_Slot(lane, torch.empty(slot_bytes, dtype=torch.uint8, device="cuda"),
                                        torch.empty(slot_bytes, dtype=torch.uint8, pin_memory=True),
                                        torch.empty(slot_bytes, dtype=torch.uint8, pin_memory=True),
                                        torch.empty(desc_bytes, dtype=torch.uint8, device="cuda"),
                                        (L.BatchItem * max_items)(), torch.cuda.Event()))
        self.slot_bytes = slot_bytes
        self.resident_bytes = sum(t.stats()["table_bytes"] for t in tables)

    def hbm_budget(self) -> dict:
        return {"resident_tables_bytes": self.resident_bytes,
                "launch_slots_bytes": sum(s.d_buf.numel() + s.desc.numel() for s in self.slots),
                "slots": len(self.slots), "slot_bytes": self.slot_bytes}

    # ------------------------------------------------------------------
    def _need(self, r: ServedRequest) -> tuple[int, int]:
        """(input bytes, output bytes) of a request inside a slot."""
        t = self.tables[r.table]
        inb = _round(r.n * t.key_bytes) + (_round(r.n * t.val_bytes) if r.op == L.OP_INSERT and t.is_map else 0)
        outb = _round(r.n) + (_round(r.n * t.val_bytes) if r.op == L.OP_FIND and t.is_map else 0)
        return inb, outb

    def _launch(self, slot: _Slot, reqs: list[ServedRequest]):
        """Stage, run and read back one launch on the slot's lane."""
        s = self.streams[slot.lane]
        sizes = [self._need(r) for r in reqs]
        in_total = sum(a for a, _ in sizes)
        layout = []
        h_in = slot.h_in.numpy()
        off = 0
        packed_end = 0
        direct = []                              # (device offset, host tensor) copied on their own
        for r, (inb, outb) in zip(reqs, sizes):
            t = self.tables[r.table]
            k_off = off
            v_off = off + _round(r.n * t.key_bytes) if (r.op == L.OP_INSERT and t.is_map) else None
            if r.n <= PACK_LIMIT:
                nb = r.n * t.key_bytes
                h_in[k_off:k_off + nb] = r.keys.numpy().view(np.uint8)[:nb]
                if v_off is not None:
                    h_in[v_off:v_off + r.n * t.val_bytes] = r.vals.numpy().view(np.uint8)
                packed_end = off + inb
            else:
                direct.append((k_off, r.keys))
                if v_off is not None:
                    direct.append((v_off, r.vals))
            layout.append((k_off, v_off))
            off += inb
        out_off = _round(in_total)
        outs = []
        o = out_off
        for r, (inb, outb) in zip(reqs, sizes):
            t = self.tables[r.table]
            v_out = o + _round(r.n) if (r.op == L.OP_FIND and t.is_map) else None
            outs.append((o, v_out))
            o += outb
        out_total = o - out_off
        d = slot.d_buf
        with torch.cuda.stream(s):
            if packed_end:
                d[:packed_end].copy_(slot.h_in[:packed_end], non_blocking=True)
            for doff, ht in direct:
                nb = ht.numel() * ht.element_size()
                d[doff:doff + nb].copy_(ht.view(torch.uint8), non_blocking=True)
            items = slot.items
            base = d.data_ptr()
            for i, r in enumerate(reqs):
                t = self.tables[r.table]
                k_off, v_off = layout[i]
                o_off, vo_off = outs[i]
                items[i] = L.BatchItem(t.handle, r.op, 0, base + k_off, base + v_off if v_off is not None else None,
                                       r.n, base + o_off, base + vo_off if vo_off is not None else None)
            if self.merge:
                L.check(self.lib.hc_batch_run(items, len(reqs), ctypes.byref(self.cfg), slot.desc.data_ptr(),
                                              slot.desc.numel(), s.cuda_stream))
            else:
                h = s.cuda_stream
                for it in items[:len(reqs)]:
                    if it.op == L.OP_INSERT:
                        L.check(self.lib.hc_insert(it.table, it.d_keys, it.d_vals, it.n, it.d_out, h))
                    elif it.op == L.OP_FIND:
                        L.check(self.lib.hc_find(it.table, it.d_keys, it.n, it.d_out, it.d_vals_out, h))
                    else:
                        L.check(self.lib.hc_erase(it.table, it.d_keys, it.n, it.d_out, h))
            slot.h_out[:out_total].copy_(d[out_off:out_off + out_total], non_blocking=True)
            ev = slot.done_event
            ev.record(s)
        slot.event = ev
        slot.reqs = reqs
        slot.layout = [(o - out_off, (vo - out_off) if vo is not None else None) for o, vo in outs]

    def _complete(self, slot: _Slot, t_done: float):
        h_out = slot.h_out.numpy()
        for r, (o, vo) in zip(slot.reqs, slot.layout):
            t = self.tables[r.table]
            r.status = h_out[o:o + r.n].copy()
            if vo is not None:
                r.values = h_out[vo:vo + r.n * t.val_bytes].copy().view(np.int32 if t.val_bytes == 4 else np.int64)
            r.done = t_done
        slot.event = None
        slot.reqs = []

    # ------------------------------------------------------------------
    def run(self, requests: list[ServedRequest], realtime: bool = True, timeout_s: float = 600.0) -> dict:
        """Serve `requests` (sorted by arrival).  With realtime=False every
        request counts as arrived at time 0 (a capacity measurement)."""
        for r in requests:
            inb, outb = self._need(r)
            if inb + outb + 256 > self.slot_bytes:
                raise ValueError(f"request {r.rid} needs {inb + outb} bytes, more than a launch slot")
        pending = deque(requests)
        fifo = [deque() for _ in self.tables]
        lane_tables = [[t for t in range(len(self.tables)) if t % self.lanes == lane] for lane in range(self.lanes)]
        rr = [0] * self.lanes
        launches = 0
        queued_max = 0
        n_done = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while n_done < len(requests):
            now = time.perf_counter() - t0
            if now > timeout_s:
                raise TimeoutError(f"served {n_done} of {len(requests)} requests in {timeout_s} s")
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                fifo[r.table].append(r)
            queued_max = max(queued_max, sum(len(f) for f in fifo))
            for slot in self.slots:
                if slot.event is not None and slot.event.query():
                    done_at = time.perf_counter() - t0
                    n_done += len(slot.reqs)
                    self._complete(slot, done_at)
            for slot in self.slots:
                if slot.event is not None:
                    continue
                lane = slot.lane
                tabs = lane_tables[lane]
                batch, used = [], 256
                cap = self.max_items if self.merge else 1
                for j in range(len(tabs)):
                    t = tabs[(rr[lane] + j) % len(tabs)]
                    if fifo[t]:
                        inb, outb = self._need(fifo[t][0])
                        if used + inb + outb > self.slot_bytes:
                            continue
                        r = fifo[t].popleft()
                        r.admitted = now
                        batch.append(r)
                        used += inb + outb
                        if len(batch) == cap:
                            break
                if batch:
                    rr[lane] = (rr[lane] + 1) % max(1, len(tabs))
                    self._launch(slot, batch)
                    launches += 1
        wall = time.perf_counter() - t0
        lat = np.array([r.done - (r.arrival if realtime else 0.0) for r in requests]) * 1e3
        ops = sum(r.n for r in requests)
        return {"requests": len(requests), "ops": ops, "wall_s": round(wall, 4), "mops": round(ops / wall / 1e6, 2),
                "launches": launches, "p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3), "p999_ms": round(float(np.percentile(lat, 99.9)), 3),
                "max_ms": round(float(lat.max()), 3), "queued_max": queued_max, "merge": self.merge,
                "lanes": self.lanes, "depth": self.depth}
