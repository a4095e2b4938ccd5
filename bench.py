"""Benchmark of the GB300 hash containers.

Default workload (one "step" = one pass of the whole hot path over one batch
of synthetic input): an unordered_map<uint64, uint64> of 2^28 slots is cleared,
filled to load factor 0.8 with uniform splitmix64 keys in batches of 2^26
(value = splitmix64(key)), then queried with 2^26 present keys and 2^26 absent
keys, then 2^26 present keys are erased.  Inputs are resident in HBM before
the timed region; the 4 GiB table is far larger than L2, so no L2 flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gpu,reference}]

Prints one JSON line.  `--impl reference` times the CPU oracle (the
single-threaded chained table) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mops/s insert/find/erase at LF 0.8; p50/p99 batch latency; % of HBM peak"
# algorithmic bytes per op for map<u64,u64>: one 32-byte slot sector read
# (+ one written for modifying ops) + key/value in + status/value out
BYTES_PER_OP = {"insert": 16 + 1 + 32 + 32, "find": 8 + 8 + 1 + 32, "erase": 8 + 1 + 32 + 32}
# DRAM bytes per op of the range insert kernel (k_insert_stream<map<u64,u64>,
# 64-byte buckets, 4 keys/thread, 2 in flight>, 64-thread blocks) on this
# workload: dram__bytes_read.sum + dram__bytes_write.sum over the four fill
# launches of one step at full size (one ncu capture), divided by the keys
# they inserted; `requests_per_op` the same for lts__t_requests_srcunit_tex.sum
# (requests from the SMs to L2).  Valid only while the kernel sources hash to
# `digest`.
INSERT_TRAFFIC = {"bytes_per_op": 227.7, "requests_per_op": 3.545, "digest": "a09fabcd81947d1e"}


def insert_kernel_digest() -> str:
    """Hash of the insert kernel's source: the device core, the streaming
    insert's chunk function and kernel with its launch bound, and its
    launcher."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_1908_05936_gb300", "csrc")
    read = lambda f: open(os.path.join(csrc, f)).read()
    stream, kernels = read("hc_stream.cuh"), read("hc_kernels.cuh")
    parts = [open(os.path.join(ROOT, "include", "hc_core.cuh")).read(),
             re.search(r"#ifndef HC_STREAM_INSERT_MINB.*?#endif", stream, re.S).group(0),
             re.search(r"template <class T, int KPT>\nstruct Stage \{.*?\n\};\n", stream, re.S).group(0),
             re.search(r"__device__ __forceinline__ void insert_stream_chunk\(.*?\n}\n", stream, re.S).group(0),
             re.search(r"template <int KIND, int BB, int KPT, int S>\n__global__[^\n]*\nk_insert_stream\(.*?\n}\n",
                       stream, re.S).group(0),
             re.search(r"cudaError_t launch_insert_stream\(.*?\n}\n", kernels, re.S).group(0)]
    return hashlib.sha256("\n".join(parts).encode()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--slots-log2", type=int, default=28)
    ap.add_argument("--batch-log2", type=int, default=26)
    ap.add_argument("--lf", type=float, default=0.8)
    ap.add_argument("--bucket-bytes", type=int, default=0, help="0 = tuned default")
    ap.add_argument("--lane-bytes", type=int, default=0)
    ap.add_argument("--kpt", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--find-lane-bytes", type=int, default=0,
                    help="lane bytes of the lookups only (the bucket size: lane-pair lookups for maps)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the batched, served, RGB-D and set<u32> comparisons")
    ap.add_argument("--cpu-sample-log2", type=int, default=24)
    ap.add_argument("--workload", default="map_sweep",
                    choices=["map_sweep", "map_grid", "device_api", "multi_table", "served", "rgbd", "set_u32",
                             "read_ceiling"])
    ap.add_argument("--rgbd-slots", type=int, default=12_500_000)
    ap.add_argument("--rgbd-hash", type=int, default=1,
                    help="1 = the paper's spatial hash on packed 21-bit coordinates, 2 = on short3 keys, 0 = mix64")
    ap.add_argument("--tables", type=int, default=1024)
    ap.add_argument("--tile", type=int, default=None,
                    help="multi_table: keys per chunk (0 = auto); no shape option = the tuned batched shape")
    ap.add_argument("--requests", type=int, default=3000)
    ap.add_argument("--served-tables", type=int, default=64)
    ap.add_argument("--served-slots", type=int, default=56_000_000)
    return ap.parse_args()


# --------------------------------------------------------------- workload --

class Workload:
    def __init__(self, slots_log2: int, batch_log2: int, lf: float, seed: int = 0):
        from workloads import recipes
        self.slots = 1 << slots_log2
        self.batch = 1 << batch_log2
        self.n_fill = recipes.fill_count(self.slots, lf)
        self.seed = seed
        self.name = (f"map<u64,u64> {self.slots} slots: fill to LF {lf} in batches of {self.batch}, "
                     f"find {self.batch} hit + {self.batch} miss, erase {self.batch}")

    def host_arrays(self):
        from workloads import recipes, splitmix
        fill = recipes.map_fill_keys(0, self.n_fill, self.seed)
        vals = splitmix.value_of(fill)
        hit = recipes.map_hit_keys(self.n_fill, self.batch, self.seed)
        miss = recipes.map_miss_keys(self.batch, self.seed, start=self.n_fill)
        er = recipes.map_hit_keys(self.n_fill, self.batch, self.seed, salt=1)
        return fill, vals, hit, miss, er

    def ops_per_step(self) -> int:
        return self.n_fill + 3 * self.batch


# ----------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi samples of SM clocks and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ replicas --

def max_over_ranks(x: float, device=None) -> float:
    """The slowest rank's time: every rank runs its own independent table (the
    units are independent, so there is no data-path collective); the job's
    time is the max over ranks, taken with one all-reduce of a scalar."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job Mops/s: the units all ranks processed over the slowest time."""
    return units_per_rank * world / (max_ms * 1e-3) / 1e6


# --------------------------------------------------------------- gpu arm --

def run_gpu(args, rank: int, world: int):
    import torch
    from paper_1908_05936_gb300 import _lib as L
    from paper_1908_05936_gb300 import build
    from paper_1908_05936_gb300.table import Table, to_device

    build.build()
    dev = torch.device("cuda", rank % max(1, torch.cuda.device_count()))
    torch.cuda.set_device(dev)
    wl = Workload(args.slots_log2, args.batch_log2, args.lf, seed=rank)
    fill, vals, hit, miss, er = wl.host_arrays()
    d_fill, d_vals, d_hit, d_miss, d_er = (to_device(a) for a in (fill, vals, hit, miss, er))
    B = wl.batch
    st_buf = torch.empty(B, dtype=torch.uint8, device=dev)
    found = torch.empty(B, dtype=torch.uint8, device=dev)
    vout = torch.empty(B, dtype=torch.int64, device=dev)

    bb = args.bucket_bytes or 64
    t = Table(L.MAP_U64_U64, wl.slots, bucket_bytes=bb)
    for op in (0, 1, 2):
        t.set_launch(op, lane_bytes=args.lane_bytes, keys_per_group=args.kpt, block=args.block)
    if args.find_lane_bytes:
        t.set_launch(1, lane_bytes=args.find_lane_bytes)
    stream = torch.cuda.current_stream()
    calls = []   # (name, n, start_event, end_event)
    in_kernel = args.workload == "device_api"
    if in_kernel:
        # the same step through a user kernel calling the in-kernel function
        # form, one operation per thread (examples/device_api.cu)
        from paper_1908_05936_gb300 import device_api as D
        build.build_examples()
        dv = t.device_view()
        blk = args.block or 128

        def do_insert(k, v, st):
            D.apply(t, k, L.OP_INSERT, vals=v, status=st, block=blk, view=dv)

        def do_find(k, f, vo):
            D.apply(t, k, L.OP_FIND, status=f, vals_out=vo, block=blk, view=dv)

        def do_erase(k, st):
            D.apply(t, k, L.OP_ERASE, status=st, block=blk, view=dv)
    else:
        def do_insert(k, v, st):
            t.insert(k, v, status=st)

        def do_find(k, f, vo):
            t.find(k, found=f, vals_out=vo)

        def do_erase(k, st):
            t.erase(k, status=st)

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def step(record: bool):
        rec = []
        e0 = ev()
        t.clear()
        e1 = ev()
        rec.append(("clear", 0, e0, e1))
        for off in range(0, wl.n_fill, B):
            n = min(B, wl.n_fill - off)
            a = ev()
            do_insert(d_fill[off:off + n], d_vals[off:off + n], st_buf[:n])
            b = ev()
            rec.append(("insert", n, a, b))
        a = ev()
        do_find(d_hit, found, vout)
        b = ev()
        rec.append(("find_hit", B, a, b))
        a = ev()
        do_find(d_miss, found, vout)
        b = ev()
        rec.append(("find_miss", B, a, b))
        a = ev()
        do_erase(d_er, st_buf)
        b = ev()
        rec.append(("erase", B, a, b))
        if record:
            calls.extend(rec)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    # correctness guard on the last warm-up step's table state
    size_after = t.size()
    expected_size = wl.n_fill - B   # fill keys are distinct with probability ~1 - 2^-10
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        step(True)
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    elapsed_ms = start.elapsed_time(end)
    elapsed_ms = max_over_ranks(elapsed_ms, dev)

    per = {}
    for name, n, a, b in calls:
        per.setdefault(name, []).append((n, a.elapsed_time(b)))
    summary = {}
    for name, lst in sorted(per.items()):
        ms = [x[1] for x in lst]
        n = sum(x[0] for x in lst)
        summary[name] = {"launches": len(lst), "ms_total": sum(ms), "p50_ms": float(np.percentile(ms, 50)),
                         "p99_ms": float(np.percentile(ms, 99))}
        if n:
            summary[name]["mops"] = n / (sum(ms) * 1e-3) / 1e6
    # insert throughput per batch position in the fill (load factor range)
    nb = len(per["insert"]) // args.steps
    lf_of = lambda i: round(min(wl.n_fill, (i + 1) * B) / wl.slots, 3)
    summary["insert_by_batch"] = [
        {"lf_end": lf_of(i), "mops": round(sum(x[0] for x in per["insert"][i::nb]) /
                                          (sum(x[1] for x in per["insert"][i::nb]) * 1e-3) / 1e6, 1)}
        for i in range(nb)]

    value = job_throughput(wl.ops_per_step() * args.steps, world, elapsed_ms)

    # roofline of the dominant kernel (largest share of the timed region)
    kinds = {"insert": "insert", "find_hit": "find", "find_miss": "find", "erase": "erase"}
    dom = max((k for k in per if k in kinds), key=lambda k: summary[k]["ms_total"])
    dom_n = sum(x[0] for x in per[dom]) / len(per[dom])
    dom_ms = summary[dom]["ms_total"] / len(per[dom])
    achieved = BYTES_PER_OP[kinds[dom]] * dom_n / (dom_ms * 1e-3) / 1e9
    traffic = None
    if (dom == "insert" and not in_kernel and bb == 64 and t.get_launch(0)["keys_per_group"] == 4
            and t.get_launch(0)["block"] == 64 and insert_kernel_digest() == INSERT_TRAFFIC["digest"]):
        traffic = INSERT_TRAFFIC["bytes_per_op"] * dom_n      # DRAM bytes per launch
    peak, peak_src = hbm_peak()
    ceiling = random_read_ceiling(torch, L)
    # the same kernel against the device's rate of scattered L2 requests
    # (random 32-byte reads, measured above): requests per op x ops per second
    requests = None
    if traffic:
        req_rate = INSERT_TRAFFIC["requests_per_op"] * dom_n / (dom_ms * 1e-3) / 1e9
        requests = {"per_op": INSERT_TRAFFIC["requests_per_op"], "achieved": round(req_rate, 1),
                    "ceiling": ceiling["reads_per_s"], "unit": "G L2 requests/s",
                    "frac": round(req_rate / ceiling["reads_per_s"], 3),
                    "source": "ncu lts__t_requests_srcunit_tex.sum, full-size capture"}

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mops/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded splitmix64 keys)",
        "config": {"workload": wl.name, "slots": wl.slots, "batch": B, "load_factor": args.lf,
                   "bucket_bytes": bb,
                   "launch": {op: t.get_launch(i) for i, op in enumerate(("insert", "find", "erase"))},
                   "l2": "inputs larger than L2 (4 GiB table)",
                   "parallelism": f"replicas{world}"},
        "ops": {k: ({kk: round(vv, 4) if isinstance(vv, float) else vv for kk, vv in v.items()}
                    if isinstance(v, dict) else v) for k, v in summary.items()},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                     "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": round(traffic) if traffic else None, "bytes_per_op": BYTES_PER_OP[kinds[dom]],
                     "dram_gbs": round(traffic / (dom_ms * 1e-3) / 1e9, 1) if traffic else None,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, full-size capture"
                     if traffic else "no capture for this kernel as built",
                     "requests": requests},
        "at_lf08": {"insert_mops": summary["insert_by_batch"][-1]["mops"],
                    "insert_batch_lf": [round(max(0.0, (nb - 1) * B / wl.slots), 3), summary["insert_by_batch"][-1]["lf_end"]],
                    "find_hit_mops": round(summary["find_hit"]["mops"], 1),
                    "find_miss_mops": round(summary["find_miss"]["mops"], 1),
                    "erase_mops": round(summary["erase"]["mops"], 1),
                    "note": "insert: the fill's last batch (load factor from..to); lookups and erase run on the "
                            "table at load factor 0.8"},
        "random_read_ceiling": ceiling,
        "clocks": clk,
        "gpu_launches": len(calls) * world,
        "check": {"size_after_step": size_after, "expected": expected_size},
    }
    if in_kernel:
        out["metric"] = "in-kernel function form: " + METRIC
        out["config"]["form"] = "user kernel, one hcd::Table call per thread (examples/device_api.cu)"
        out["config"]["launch"] = {"block": blk}
    else:
        out["other_ops"] = time_rehash_dump(t, torch)
        out["other_ops"]["ordered_mixed"] = time_ordered_mixed(t, torch, seed=rank)
    if not args.no_e2e and not in_kernel:
        out["e2e"] = run_e2e(t, wl, fill, vals, hit, miss, er, stream)
    t.close()
    return out


def time_rehash_dump(t, torch):
    """Host-called whole-table operations on the table a step left behind
    (load factor 0.55 plus the step's tombstones), timed once each by wall
    clock (both synchronise): rehash to the same capacity, which purges the
    tombstones, then dump of every stored pair, and size."""
    torch.cuda.synchronize()
    st0 = t.stats()
    t0 = time.perf_counter()
    t.rehash(st0["capacity"])
    rehash_s = time.perf_counter() - t0
    st1 = t.stats()
    t0 = time.perf_counter()
    k, v = t.dump()
    torch.cuda.synchronize()
    dump_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    live = t.size()
    size_s = time.perf_counter() - t0
    assert len(k) == live == st1["live"] == st0["live"]
    del k, v
    # selection of about 1/16 of the entries (keys below 2^60), timed with
    # CUDA events: one pass over every slot's key, values of the matches
    from paper_1908_05936_gb300 import _lib as L
    ko = torch.empty(live // 8, dtype=torch.int64, device="cuda")
    vo = torch.empty(live // 8, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    t.select(L.PRED_KEY_RANGE, 0, 2**60 - 1, keys_out=ko, vals_out=vo, count=cnt)
    ms = []
    for _ in range(5):
        cnt.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        t.select(L.PRED_KEY_RANGE, 0, 2**60 - 1, keys_out=ko, vals_out=vo, count=cnt)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    sel = int(cnt.item())
    sel_ms = float(np.median(ms))
    key_bytes = st1["capacity"] * 8          # every slot's key is read once
    del ko, vo
    return {"rehash": {"ms": round(rehash_s * 1e3, 2), "live": st0["live"], "used_before": st0["used"],
                       "used_after": st1["used"], "mkeys_per_s": round(st0["live"] / rehash_s / 1e6, 1)},
            "dump": {"ms": round(dump_s * 1e3, 2), "mkeys_per_s": round(live / dump_s / 1e6, 1)},
            "select": {"ms": round(sel_ms, 3), "selected": sel, "slots_per_s_g": round(st1["capacity"] / sel_ms / 1e6, 1),
                       "key_gbs": round((key_bytes + sel * 32) / (sel_ms * 1e-3) / 1e9, 1)},
            "size": {"us": round(size_s * 1e6, 1)}}


def time_ordered_mixed(t, torch, seed: int = 0) -> dict:
    """Ordered calls and mixed batches on the table a step left behind
    (rehashed), against the plain calls on the same keys; CUDA events, median
    of three repetitions, nothing here inside the step's timed region.

    * ordered insert / erase (the lowest index wins among equal keys, every
      position gets the sequential result) of 2^24 draws from 2^23 fresh keys
      (at most capacity / 16 draws on smaller tables),
      against the plain insert / erase of the same draws;
    * a free-running mixed batch over the same draws (50 / 30 / 20 insert /
      find / erase, per position), against the three plain calls of its parts.
    Every repetition starts from the same table: after each timed call that
    inserts the draws' keys they are erased and the table is rehashed to its
    own capacity (both untimed), so tombstones of earlier repetitions do not
    lengthen the probes of later ones (the mixed batch's inserts claim EMPTY
    slots only and would otherwise use up a few million per repetition)."""
    from paper_1908_05936_gb300.table import to_device
    from workloads import recipes, splitmix
    # 2^24 draws from 2^23 keys on the 2^28-slot table; fewer on smaller
    # tables: the mixed batch's in-kernel inserts claim EMPTY slots only, so
    # its repetitions must leave the table most of its EMPTY slots
    cap = t.stats()["capacity"]
    n = 1 << 24
    while n > 1024 and n > cap // 16:
        n >>= 1
    nd = n // 2
    keys_h = recipes.repeated_keys(n, nd, seed)
    ops_h = recipes.mixed_ops(n, seed=seed)
    d_keys, d_vals = to_device(keys_h), to_device(splitmix.value_of(keys_h))
    d_ops = torch.from_numpy(ops_h).cuda()
    d_parts = [to_device(keys_h[ops_h == k]) for k in range(3)]
    d_part_vals = to_device(splitmix.value_of(keys_h[ops_h == 0]))
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    vo = torch.empty(n, dtype=torch.int64, device="cuda")
    scratch = torch.empty(int(t.lib.hc_ordered_scratch_bytes(n)) + 256, dtype=torch.uint8, device="cuda")
    live0 = t.size()

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    def reset():
        t.erase(d_keys, status=False)
        t.rehash(cap)
        torch.cuda.synchronize()

    res = {k: [] for k in ("insert", "insert_ordered", "erase", "erase_ordered", "mixed", "parts")}
    for _ in range(4):
        res["insert"].append(timed(lambda: t.insert(d_keys, d_vals, status=st)))
        res["erase"].append(timed(lambda: t.erase(d_keys, status=st)))
        t.rehash(cap)
        res["insert_ordered"].append(timed(lambda: t.insert_ordered(d_keys, d_vals, status=st, scratch=scratch)))
        res["erase_ordered"].append(timed(lambda: t.erase_ordered(d_keys, status=st, scratch=scratch)))
        t.rehash(cap)
        res["mixed"].append(timed(lambda: t.apply_mixed(d_ops, d_keys, d_vals, status=st, vals_out=vo)))
        reset()

        def parts():
            t.insert(d_parts[0], d_part_vals, status=st)
            t.find(d_parts[1], found=st, vals_out=vo)
            t.erase(d_parts[2], status=st)
        res["parts"].append(timed(parts))
        reset()
    assert t.size() == live0
    med = {k: float(np.median(v[1:])) for k, v in res.items()}        # the first repetition warms up
    rate = lambda ms: round(n / (ms * 1e-3) / 1e6, 1)
    return {"keys": n, "distinct": nd, "mix": [0.5, 0.3, 0.2],
            **{k: {"ms": round(v, 3), "mops": rate(v)} for k, v in med.items()},
            "ordered_over_plain": {"insert": round(med["insert_ordered"] / med["insert"], 2),
                                   "erase": round(med["erase_ordered"] / med["erase"], 2)},
            "mixed_over_parts": round(med["mixed"] / med["parts"], 2)}


def run_e2e(t, wl, fill, vals, hit, miss, er, stream):
    """Same step through the C ABI's host-buffer calls: page-locked host
    arrays in, host results out, every transfer inside the timed region (the
    kernels read and write the page-locked arrays in place)."""
    import torch
    pin = lambda a: torch.from_numpy(a.view(np.int64)).pin_memory().numpy().view(a.dtype)
    fill_p, vals_p, hit_p, miss_p, er_p = (pin(a) for a in (fill, vals, hit, miss, er))
    st = torch.empty(wl.n_fill, dtype=torch.uint8).pin_memory().numpy()
    fnd = torch.empty(wl.batch, dtype=torch.uint8).pin_memory().numpy()
    vo = torch.empty(wl.batch, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
    est = torch.empty(wl.batch, dtype=torch.uint8).pin_memory().numpy()

    def step():
        t.clear()
        t.insert_host(fill_p, vals_p, st)
        t.find_host(hit_p, fnd, vo)
        t.find_host(miss_p, fnd, vo)
        t.erase_host(er_p, est)

    step()
    torch.cuda.synchronize()
    reps = 2
    t0 = time.perf_counter()
    for _ in range(reps):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    h2d = fill.nbytes + vals.nbytes + hit.nbytes + miss.nbytes + er.nbytes
    d2h = wl.n_fill + 2 * (wl.batch * 9) + wl.batch
    return {"value": round(wl.ops_per_step() / dt / 1e6, 2), "unit": "Mops/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": round(dt * 1e3, 2),
            "transfer": "page-locked host arrays, read and written in place by the kernels (NVLink-C2C)"}


def random_read_ceiling(torch, L):
    """Measured rate of random 32-byte reads over a 2 GiB buffer (larger than
    L2): the ceiling of a probe-bound operation on this device."""
    import ctypes
    buf = torch.empty(1 << 31, dtype=torch.uint8, device="cuda")
    ms = ctypes.c_float()
    n = 1 << 26
    L.check(L.load().hc_measure_random_reads(buf.data_ptr(), buf.numel(), n, 5, ctypes.byref(ms),
                                             torch.cuda.current_stream().cuda_stream))
    del buf
    rate = n / (ms.value * 1e-3)
    return {"reads_per_s": round(rate / 1e9, 2), "unit": "G random 32-byte reads/s",
            "line_traffic_gbs": round(rate * 128 / 1e9, 1),
            "note": "each random read moves one 128-byte line from HBM on this GPU"}


def run_read_ceiling(args):
    """Calibration: the rate of random 32-byte reads (hc_measure_random_reads,
    2^26 reads per launch, five launches after one warm-up) over buffers from
    8 MiB (inside L2) to 16 GiB.  Beyond L2 it is the ceiling of a
    probe-bound operation."""
    import ctypes
    import torch
    from paper_1908_05936_gb300 import _lib as L
    from paper_1908_05936_gb300 import build
    build.build()
    rows = []
    for mib in (8, 32, 64, 96, 128, 256, 512, 1024, 2048, 4096, 8192, 16384):
        buf = torch.empty(mib << 20, dtype=torch.uint8, device="cuda")
        ms = ctypes.c_float()
        n = 1 << 26
        L.check(L.load().hc_measure_random_reads(buf.data_ptr(), buf.numel(), n, 5, ctypes.byref(ms),
                                                 torch.cuda.current_stream().cuda_stream))
        del buf
        torch.cuda.empty_cache()
        rows.append({"buffer_mib": mib, "g_reads_per_s": round(n / (ms.value * 1e-3) / 1e9, 2)})
    return {"metric": "random 32-byte reads per second by buffer size", "value": rows[9]["g_reads_per_s"],
            "unit": "G reads/s (4 GiB)", "n_gpus": 1, "higher_is_better": True, "dtype": "u8",
            "data": "synthetic (pseudo-random offsets)", "config": {"workload": "calibration, 2^26 reads per launch"},
            "sweep": rows}


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def bytes_fraction(total_bytes: float, ms: float, per_op: dict, note: str) -> dict:
    """Algorithmic bytes of a whole step (per-op minimum bytes x ops) over
    its measured time, against the measured copy peak."""
    peak, src = hbm_peak()
    gbs = total_bytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "peak_source": src, "unit": "GB/s",
            "frac": round(gbs / peak, 4), "bytes_per_op": per_op, "traffic": None, "note": note}


# ---------------------------------------------------------- oracle (CPU) --

def run_oracle_sample(args, sample_log2: int):
    """The CPU oracle, as it stands, on a bounded sample of the workload:
    fill 2^sample keys into a table of the same capacity semantics, then
    2^(sample-2) present finds, absent finds and erases."""
    from oracle import oracle as O
    from workloads import recipes, splitmix
    n = 1 << sample_log2
    q = n // 4
    fill = recipes.map_fill_keys(0, n)
    vals = splitmix.value_of(fill)
    hit = recipes.map_hit_keys(n, q)
    miss = recipes.map_miss_keys(q, start=n)
    er = recipes.map_hit_keys(n, q, salt=1)
    t = O.OracleTable(O.MAP_U64_U64, 1 << args.slots_log2)
    per = {}
    t0 = time.perf_counter()
    for name, fn, cnt in (("insert", lambda: t.insert(fill, vals), n), ("find_hit", lambda: t.find(hit), q),
                          ("find_miss", lambda: t.find(miss), q), ("erase", lambda: t.erase(er), q)):
        a = time.perf_counter()
        fn()
        per[name] = round(cnt / (time.perf_counter() - a) / 1e6, 3)
    dt = time.perf_counter() - t0
    t.close()
    ops = n + 3 * q
    return {"value": round(ops / dt / 1e6, 3), "unit": "Mops/s", "cores": 1, "kind": "oracle",
            "sample": f"fill {n} keys, find {q} hit + {q} miss, erase {q} (single-threaded C chained table)",
            "seconds": round(dt, 2), "ops_mops": per, "host_cores_available": os.cpu_count(),
            "host_cpu": host_cpu()}


def host_cpu() -> str:
    """The host CPU's model name (lscpu), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


# ------------------------------------------------ multi-table workload --

def run_multi_table(args):
    """1024 set<u64> tables, capacities log-uniform in 2^10..2^22; each gets
    0.5 x capacity ops (60 % insert, 30 % find, 10 % erase).  The plain form
    is 3 x 1024 range calls; the batched form is one CUDA graph of three
    persistent phase kernels.  A step is the op batch of every table; the
    tables are cleared between steps, outside the timed intervals."""
    import torch
    from paper_1908_05936_gb300 import _lib as L
    from paper_1908_05936_gb300 import build
    from paper_1908_05936_gb300.batch import Batch, Item
    from paper_1908_05936_gb300.table import Table, to_device
    from workloads import recipes

    build.build()
    n_tables = args.tables
    slots = recipes.multi_table_slots(n_tables)
    ops = [recipes.multi_table_ops(int(s), t) for t, s in enumerate(slots)]
    n_ops = sum(len(o.insert_keys) + len(o.find_keys) + len(o.erase_keys) for o in ops)
    from paper_1908_05936_gb300 import tune
    shape = None
    if not (args.bucket_bytes or args.lane_bytes or args.kpt or args.block or args.tile is not None):
        shape = tune.batch_config()                   # the autotuner's choice on this GPU, if cached
    source = "tuned (tune.py --batch)" if shape else "arguments"
    if shape is None:
        shape = dict(bucket_bytes=args.bucket_bytes or 128, lane_bytes=args.lane_bytes, keys_per_group=args.kpt,
                     block=args.block, tile=args.tile if args.tile is not None else 4096)
    bb = shape["bucket_bytes"]
    arms = {}
    for arm in ("plain", "batched"):
        tabs = [Table(L.SET_U64, int(s), bucket_bytes=bb) for s in slots]
        items = []
        for t, o in zip(tabs, ops):
            ki, kf, ke = to_device(o.insert_keys), to_device(o.find_keys), to_device(o.erase_keys)
            items += [Item(t, L.OP_INSERT, ki, None, torch.empty(ki.numel(), dtype=torch.uint8, device="cuda")),
                      Item(t, L.OP_FIND, kf, None, torch.empty(kf.numel(), dtype=torch.uint8, device="cuda")),
                      Item(t, L.OP_ERASE, ke, None, torch.empty(ke.numel(), dtype=torch.uint8, device="cuda"))]
        batch = Batch(items, lane_bytes=shape["lane_bytes"], keys_per_group=shape["keys_per_group"],
                      block=shape["block"], tile=shape["tile"], use_graph=True) if arm == "batched" else None
        stream = torch.cuda.current_stream()

        def step():
            if batch is not None:
                batch.launch()
                return 3
            for it in items:
                if it.op == L.OP_INSERT:
                    it.table.insert(it.keys, None, status=it.out)
                elif it.op == L.OP_FIND:
                    it.table.find(it.keys, found=it.out, vals_out=False)
                else:
                    it.table.erase(it.keys, status=it.out)
            return len(items)

        times, launches = [], 0
        for i in range(args.warmup + args.steps):
            for t in tabs:
                t.clear()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            nl = step()
            b.record(stream)
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(a.elapsed_time(b))
                launches += nl
        sizes = sum(t.size() for t in tabs)
        arms[arm] = {"ms_per_step": round(statistics.median(times), 3), "mops": round(n_ops / statistics.median(times) / 1e3, 1),
                     "launches_per_step": launches // args.steps, "live_after": sizes}
        for t in tabs:
            t.close()
        if batch is not None:
            batch.close()
        del items
        torch.cuda.empty_cache()
    assert arms["plain"]["live_after"] == arms["batched"]["live_after"], "plain and batched forms disagree"
    per_op = {"insert": 8 + 1 + 32 + 32, "find": 8 + 1 + 32, "erase": 8 + 1 + 32 + 32}
    step_bytes = sum(len(o.insert_keys) * per_op["insert"] + len(o.find_keys) * per_op["find"] +
                     len(o.erase_keys) * per_op["erase"] for o in ops)
    return {"metric": "multi-table batched vs plain: ms per step and Mops/s", "value": arms["batched"]["mops"],
            "unit": "Mops/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": arms["batched"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded splitmix64 keys)",
            "config": {"workload": f"{n_tables} set<u64> tables, capacities round(2^U(10,22)), 0.5 x capacity ops "
                                   "60/30/10 insert/find/erase", "total_slots": int(slots.sum()), "ops_per_step": n_ops,
                       "bucket_bytes": bb, "batch_shape": dict(shape, source=source)},
            "plain": arms["plain"], "batched": arms["batched"],
            "speedup": round(arms["plain"]["ms_per_step"] / arms["batched"]["ms_per_step"], 3),
            "roofline": bytes_fraction(step_bytes, arms["batched"]["ms_per_step"], per_op,
                                       "whole batched launch (three phase kernels); many tables are L2-resident"),
            "gpu_launches": arms["batched"]["launches_per_step"] * args.steps}


# ---------------------------------------------------- set<u32> workload --

def run_set_u32(args):
    """set<u32>, 2^21 slots (8 MiB of keys: the table lives in L2): insert
    10^6 uniform keys, find 10^6 (half present), erase 5*10^5.  A step is
    clear + the three calls; inputs stay resident; each step's calls are timed
    with CUDA events and the L2 is flushed (a 256 MiB write) between steps so
    every step starts cold."""
    import torch
    from paper_1908_05936_gb300 import _lib as L
    from paper_1908_05936_gb300 import build
    from paper_1908_05936_gb300.table import Table, to_device
    from workloads import recipes

    build.build()
    w = recipes.set_u32_workload()
    # 32-byte buckets: the fastest of 32 / 64 / 128 for this L2-resident table
    t = Table(L.SET_U32, w.slots, bucket_bytes=args.bucket_bytes or 32)
    for op in (0, 1, 2):
        t.set_launch(op, lane_bytes=args.lane_bytes, keys_per_group=args.kpt, block=args.block)
    ki, kf, ke = to_device(w.insert_keys), to_device(w.find_keys), to_device(w.erase_keys)
    si = torch.empty(ki.numel(), dtype=torch.uint8, device="cuda")
    ff = torch.empty(kf.numel(), dtype=torch.uint8, device="cuda")
    se = torch.empty(ke.numel(), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    per = {"clear": [], "insert": [], "find": [], "erase": [], "step": []}
    s = torch.cuda.current_stream()
    for i in range(args.warmup + args.steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(s)
        t.clear()
        ev[1].record(s)
        t.insert(ki, status=si)
        ev[2].record(s)
        t.find(kf, found=ff, vals_out=False)
        ev[3].record(s)
        t.erase(ke, status=se)
        ev[4].record(s)
        torch.cuda.synchronize()
        if i >= args.warmup:
            for j, k in enumerate(("clear", "insert", "find", "erase")):
                per[k].append(ev[j].elapsed_time(ev[j + 1]))
            per["step"].append(ev[0].elapsed_time(ev[4]))
    n = {"insert": ki.numel(), "find": kf.numel(), "erase": ke.numel()}
    per_op = {"insert": 4 + 1 + 32 + 32, "find": 4 + 1 + 32, "erase": 4 + 1 + 32 + 32}
    med = {k: statistics.median(v) for k, v in per.items()}
    ops = sum(n.values())
    size = t.size()
    launch = {op: t.get_launch(i) for i, op in enumerate(("insert", "find", "erase"))}
    bucket_bytes = t.bucket_bytes
    t.close()
    return {"metric": "set<u32> (L2-resident) Mops/s per op", "value": round(ops / med["step"] / 1e3, 1),
            "unit": "Mops/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(med["step"], 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic (seeded splitmix64 keys)",
            "config": {"workload": "set<u32> 2^21 slots: insert 1,000,000, find 1,000,000 (50% present), erase 500,000",
                       "l2": "256 MiB flush before each step", "bucket_bytes": bucket_bytes, "launch": launch},
            "ops": {k: {"ms": round(med[k], 4), "mops": round(n[k] / med[k] / 1e3, 1)} for k in n},
            "roofline": bytes_fraction(sum(n[k] * per_op[k] for k in n), med["step"], per_op,
                                       "the 8 MiB table is L2-resident: L2, not HBM, bounds it"),
            "clear_ms": round(med["clear"], 4), "final_size": size, "gpu_launches": 4 * args.steps}


# ---------------------------------------- load-factor x batch-size grid --

def run_map_grid(args):
    """map<u64,u64>, 2^28 slots: for every batch size 2^16 .. 2^26 and load
    factor 0.5 / 0.7 / 0.8 / 0.9, clear, fill to the load factor in batches of
    that size, then find 2^26 present and 2^26 absent keys and erase 2^26
    present keys (one call each).  CUDA events around every call; the 4 GiB
    table is far larger than L2.  Prints one line with the whole grid."""
    import torch
    from paper_1908_05936_gb300 import _lib as L
    from paper_1908_05936_gb300 import build
    from paper_1908_05936_gb300.table import Table
    from workloads import gpu as G
    from workloads import recipes

    build.build()
    slots = 1 << args.slots_log2
    q = 1 << 26
    n_max = recipes.fill_count(slots, 0.9)
    fill = G.stream_u64(3, 0, 0, n_max)
    vals = G.value_of(fill)
    miss = G.stream_u64(4, 0, 0, q)
    gen = torch.Generator(device="cuda").manual_seed(11)
    st = torch.empty(q, dtype=torch.uint8, device="cuda")
    vo = torch.empty(q, dtype=torch.int64, device="cuda")
    t = Table(L.MAP_U64_U64, slots, bucket_bytes=args.bucket_bytes or 64)
    for op in (0, 1, 2):
        t.set_launch(op, lane_bytes=args.lane_bytes, keys_per_group=args.kpt, block=args.block)
    s = torch.cuda.current_stream()

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        return a, b

    grid = []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for blog in (16, 18, 20, 22, 24, 26):
        B = 1 << blog
        for lf in (0.5, 0.7, 0.8, 0.9):
            n = recipes.fill_count(slots, lf)
            t.clear()
            torch.cuda.synchronize()
            ins = []
            for off in range(0, n, B):
                m = min(B, n - off)
                ins.append((m, *timed(lambda: t.insert(fill[off:off + m], vals[off:off + m], status=st[:m]))))
            hit = fill[torch.randperm(n, device="cuda", generator=gen)[:q]]
            fh = timed(lambda: t.find(hit, found=st, vals_out=vo))
            fm = timed(lambda: t.find(miss, found=st, vals_out=vo))
            er = timed(lambda: t.erase(hit, status=st))
            torch.cuda.synchronize()
            ins_ms = sum(a.elapsed_time(b) for _, a, b in ins)
            grid.append({"batch": B, "load_factor": lf, "insert_gops": round(n / ins_ms / 1e6, 2),
                         "insert_launches": len(ins), "find_hit_gops": round(q / fh[0].elapsed_time(fh[1]) / 1e6, 2),
                         "find_miss_gops": round(q / fm[0].elapsed_time(fm[1]) / 1e6, 2),
                         "erase_gops": round(q / er[0].elapsed_time(er[1]) / 1e6, 2),
                         "size_ok": t.size() == n - q})
    clk = clocks.stop()
    t.close()
    head = [g for g in grid if g["batch"] == 1 << 26 and g["load_factor"] == 0.8][0]
    return {"metric": "insert / find / erase G ops/s over load factor and batch size", "value": head["insert_gops"],
            "unit": "G ops/s (insert, LF 0.8, batch 2^26)", "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded splitmix64 keys)",
            "config": {"workload": f"map<u64,u64> {slots} slots, LF 0.5/0.7/0.8/0.9 x batches 2^16..2^26, "
                                   "find 2^26 present + 2^26 absent, erase 2^26",
                       "l2": "inputs larger than L2 (4 GiB table)"},
            "grid": grid, "clocks": clk}


# ------------------------------------------------------ RGB-D workload --

def rgbd_frames(params, workers: int = 8):
    """All frames' candidate keys and values (host), generated by a process
    pool started with spawn (safe next to an initialised CUDA context)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from workloads import rgbd
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        keys = list(ex.map(_rgbd_frame, [(params, f) for f in range(params.frames)], chunksize=4))
    return keys, [rgbd.values_of(k) for k in keys]


def _rgbd_frame(arg):
    from workloads import rgbd
    params, f = arg
    return rgbd.frame_keys(params, f)


def run_rgbd(args):
    """map<int64 packed block, int32>: 300 frames x 400k candidate blocks of
    the synthetic RGB-D stream; per frame, find the candidates and insert the
    missing ones.  Eager (two launches per frame) against one CUDA graph
    holding the whole stream."""
    import torch
    from paper_1908_05936_gb300 import _lib as L
    from paper_1908_05936_gb300 import build
    from paper_1908_05936_gb300.table import Table, to_device
    from workloads import rgbd

    build.build()
    params = rgbd.RGBDParams()
    t0 = time.perf_counter()
    keys, vals = rgbd_frames(params, workers=min(16, os.cpu_count() or 4))
    gen_s = time.perf_counter() - t0
    capacity = args.rgbd_slots
    # 128-byte buckets: the fastest of 32 / 64 / 128 for this stream (mostly present lookups)
    tab = Table(L.MAP_I64_I32, capacity, bucket_bytes=args.bucket_bytes or 128, hash_mode=args.rgbd_hash)
    if args.rgbd_hash == L.HASH_TESCHNER_SHORT3:
        # the paper's short3 block keys: coordinates repacked into 16-bit fields on the device
        from paper_1908_05936_gb300.table import pack_short3

        def as_short3(k):
            u = k.view(np.uint64)
            c = np.stack([((u >> np.uint64(21 * f)) & np.uint64(0x1FFFFF)).astype(np.int64) for f in range(3)], 1)
            c = np.where(c >= (1 << 20), c - (1 << 21), c).astype(np.int16)
            return pack_short3(torch.from_numpy(np.ascontiguousarray(c)).cuda())
        d_keys = [as_short3(k) for k in keys]
    else:
        d_keys = [to_device(k) for k in keys]
    d_vals = [to_device(v) for v in vals]
    found = [torch.empty(len(k), dtype=torch.uint8, device="cuda") for k in keys]
    status = [torch.empty(len(k), dtype=torch.uint8, device="cuda") for k in keys]

    def stream_all():
        for f in range(params.frames):
            tab.find(d_keys[f], found=found[f], vals_out=False)
            tab.insert_if_absent(d_keys[f], d_vals[f], found[f], status=status[f])

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        stream_all()
    res = {}
    for arm in ("eager", "graph"):
        times = []
        for i in range(args.warmup + args.steps):
            tab.clear()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            if arm == "graph":
                g.replay()
            else:
                stream_all()
            b.record()
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(a.elapsed_time(b))
        ms = statistics.median(times)
        res[arm] = {"ms_per_stream": round(ms, 3), "ms_per_frame": round(ms / params.frames, 4),
                    "mcandidates_per_s": round(params.frames * params.per_frame / ms / 1e3, 1)}
    final = tab.size()
    pres = [float(found[f].float().mean()) for f in range(params.frames)]
    tab.close()
    # every candidate is looked up; the missing ones (the table's final size) are inserted
    per_op = {"find": 8 + 4 + 1 + 32, "insert": 8 + 4 + 1 + 32 + 32}
    step_bytes = params.frames * params.per_frame * per_op["find"] + final * per_op["insert"]
    return {"metric": "RGB-D stream: per-frame find-then-insert time and candidates/s",
            "value": res["graph"]["mcandidates_per_s"], "unit": "M candidates/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["graph"]["ms_per_stream"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i64/i32",
            "data": "synthetic RGB-D voxel-block stream (sphere + planes, seeded)",
            "config": {"workload": f"map<i64,i32> {capacity} slots, {params.frames} frames x {params.per_frame} "
                                   "candidate blocks, find then insert missing", "hash_mode": args.rgbd_hash,
                       "bucket_bytes": args.bucket_bytes or 128,
                       "generation_s": round(gen_s, 1)},
            "eager": res["eager"], "graph": res["graph"], "final_blocks": final,
            "roofline": bytes_fraction(step_bytes, res["graph"]["ms_per_stream"], per_op,
                                       "find of every candidate, insert of the missing ones (graph)"),
            "final_load_factor": round(final / capacity, 4), "present_mean": round(float(np.mean(pres[1:])), 4),
            "gpu_launches": 2 * params.frames}


# ---------------------------------------------------- served workload --

def run_served(args):
    """64 resident map<u64,u64> tables (56M slots each, ~57 GB), prefilled to
    load factor 0.5; Poisson arrivals of insert/find/erase requests (40/50/10)
    with sizes floor(2^U(0,20)) and Zipf(1.1) keys over 2^24 ranks per table.
    First each form serves every request as fast as it can (its capacity:
    the median of three passes after an untimed one); then both serve
    real-time arrivals at 50 %, 80 % and 100 % of the plain path's capacity,
    fifteen runs each (medians over the runs reported: a third or more of the
    runs of either form can show a pause of tens of ms of the loop's host
    thread on the shared host, and a median over nine runs was sometimes such
    a run)."""
    import torch
    from paper_1908_05936_gb300 import _lib as L
    from paper_1908_05936_gb300 import build
    from paper_1908_05936_gb300.serve import Server, ServedRequest
    from paper_1908_05936_gb300.table import Table
    from workloads import gpu as G
    from workloads import recipes

    build.build()
    n_tables, slots = args.served_tables, args.served_slots
    tabs = [Table(L.MAP_U64_U64, slots, bucket_bytes=args.bucket_bytes or 64) for _ in range(n_tables)]
    prefill = slots // 2
    for t, tab in enumerate(tabs):
        for off in range(0, prefill, 1 << 26):
            k = G.stream_u64(7000 + t, 0, off, min(1 << 26, prefill - off))
            tab.insert(k, G.value_of(k), status=False)
    torch.cuda.synchronize()
    base = recipes.served_requests(args.requests, n_tables, 1.0)
    cdf = torch.from_numpy(recipes.zipf_cdf(1 << 24)).cuda()
    total = sum(q.n for q in base)
    keys_h = torch.empty(total, dtype=torch.int64, pin_memory=True)
    vals_h = torch.empty(total, dtype=torch.int64, pin_memory=True)
    off = 0
    spans = []
    for q in base:
        k = G.zipf_keys(q.table, q.key_stream, q.n, cdf)
        keys_h[off:off + q.n].copy_(k)
        if q.op == L.OP_INSERT:
            vals_h[off:off + q.n].copy_(G.value_of(k))
        spans.append((off, q.n))
        off += q.n
    torch.cuda.synchronize()

    def requests(rate):
        return [ServedRequest(q.rid, q.table, q.op, keys_h[o:o + n], vals_h[o:o + n] if q.op == L.OP_INSERT else None,
                              q.arrival / rate) for q, (o, n) in zip(base, spans)]

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    plain = Server(tabs, lanes=4, depth=2, merge=False)
    merged = Server(tabs, lanes=4, depth=2, merge=True)
    # capacity: every request counted as arrived at once; one untimed pass
    # per form, then the median of three (a pass lasts only tens of ms)
    def capacity(srv):
        srv.run(requests(1.0), realtime=False)
        runs = sorted((srv.run(requests(1.0), realtime=False) for _ in range(3)), key=lambda r: r["mops"])
        return dict(runs[1], mops_runs=[r["mops"] for r in runs])
    cap = capacity(plain)
    cap_rate = cap["requests"] / cap["wall_s"]
    cap_merged = capacity(merged)
    # each load point fifteen times per form, alternating; p50, p99 and Mops/s
    # are the medians over the runs (a p99 of 3000 requests rests on 30 of
    # them, and the loop's single host thread shares the host: a run whose
    # thread is held off the CPU for tens of ms shows it in every figure)
    def median_run(runs):
        med = lambda k: statistics.median(r[k] for r in runs)
        return dict(runs[0], p50_ms=med("p50_ms"), p99_ms=med("p99_ms"), mops=med("mops"),
                    p99_runs=sorted(r["p99_ms"] for r in runs), p50_runs=sorted(r["p50_ms"] for r in runs))
    loads = {}
    for frac in (0.5, 0.8, 1.0):
        rate = frac * cap_rate
        runs = {"plain": [], "merged": []}
        for _ in range(15):
            runs["plain"].append(plain.run(requests(rate), realtime=True))
            runs["merged"].append(merged.run(requests(rate), realtime=True))
        loads[f"{int(frac * 100)}%"] = {"rate_req_per_s": round(rate, 1), "plain": median_run(runs["plain"]),
                                        "merged": median_run(runs["merged"])}
    clk = clocks.stop()
    budget = merged.hbm_budget()
    for t in tabs:
        t.close()
    head = loads["80%"]
    return {"metric": "served p50/p99 latency and Mops/s vs the plain one-launch-per-request path",
            "value": head["merged"]["mops"], "unit": "Mops/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded Poisson arrivals, Zipf(1.1) keys)",
            "config": {"workload": f"{n_tables} map<u64,u64> x {slots} slots, prefilled to LF 0.5, {args.requests} "
                                   "requests, sizes floor(2^U(0,20)), 40/50/10 insert/find/erase, Zipf(1.1) over 2^24",
                       "ops": total, "hbm": budget},
            "capacity": {"plain": cap, "merged": cap_merged, "plain_req_per_s": round(cap_rate, 1)},
            "loads": loads, "clocks": clk}


def run_extras(args) -> dict:
    """The other configurations, each after the timed region of the headline
    step and outside it: the batched form against per-table launches, the
    served form against one launch per request, the RGB-D stream, and the
    L2-resident set<u32> workload.  Compact summaries; a workload that fails
    reports its error instead of ending the run."""
    import copy
    import torch
    res = {}
    for name, fn, pick in (("multi_table", run_multi_table, _pick_multi), ("served", run_served, _pick_served),
                           ("rgbd", run_rgbd, _pick_rgbd), ("set_u32", run_set_u32, _pick_set_u32)):
        a = copy.copy(args)
        a.workload = name
        t0 = time.perf_counter()
        try:
            res[name] = pick(fn(a))
        except Exception as e:                     # reported, not fatal: the headline line stands
            res[name] = {"error": f"{type(e).__name__}: {e}"}
        res[name]["wall_s"] = round(time.perf_counter() - t0, 1)
        torch.cuda.empty_cache()
    return res


def _pick_multi(r):
    return {"config": r["config"]["workload"], "shape": r["config"]["batch_shape"],
            "plain_ms": r["plain"]["ms_per_step"], "batched_ms": r["batched"]["ms_per_step"],
            "speedup": r["speedup"], "batched_mops": r["batched"]["mops"], "plain_mops": r["plain"]["mops"],
            "launches": {"plain": r["plain"]["launches_per_step"], "batched": r["batched"]["launches_per_step"]},
            "same_size": r["plain"]["live_after"] == r["batched"]["live_after"],
            "roofline_frac": r["roofline"]["frac"]}


def _pick_served(r):
    cap = r["capacity"]
    return {"config": r["config"]["workload"],
            "capacity_mops": {"plain": cap["plain"]["mops"], "merged": cap["merged"]["mops"]},
            "capacity_launches": {"plain": cap["plain"]["launches"], "merged": cap["merged"]["launches"]},
            "latency_ms": {load: {form: {"p50": v[form]["p50_ms"], "p99": v[form]["p99_ms"], "mops": v[form]["mops"],
                                         "p99_runs": v[form]["p99_runs"]}
                                  for form in ("plain", "merged")} | {"rate_req_per_s": v["rate_req_per_s"]}
                           for load, v in r["loads"].items()},
            "note": "medians over fifteen runs per load point and form; p99_runs lists every run",
            "clocks": r["clocks"]}


def _pick_rgbd(r):
    return {"config": r["config"]["workload"], "ms_per_frame": {"eager": r["eager"]["ms_per_frame"],
                                                                "graph": r["graph"]["ms_per_frame"]},
            "mcandidates_per_s": r["graph"]["mcandidates_per_s"], "final_blocks": r["final_blocks"],
            "final_load_factor": r["final_load_factor"], "present_mean": r["present_mean"],
            "roofline_frac": r["roofline"]["frac"]}


def _pick_set_u32(r):
    return {"config": r["config"]["workload"], "mops": {k: v["mops"] for k, v in r["ops"].items()},
            "ms": {k: v["ms"] for k, v in r["ops"].items()}, "final_size": r["final_size"],
            "note": r["roofline"]["note"]}


def main():
    args = parse()
    if args.workload == "multi_table":
        print(json.dumps(run_multi_table(args)))
        return
    if args.workload == "served":
        print(json.dumps(run_served(args)))
        return
    if args.workload == "rgbd":
        print(json.dumps(run_rgbd(args)))
        return
    if args.workload == "set_u32":
        print(json.dumps(run_set_u32(args)))
        return
    if args.workload == "map_grid":
        print(json.dumps(run_map_grid(args)))
        return
    if args.workload == "read_ceiling":
        print(json.dumps(run_read_ceiling(args)))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return
        wl = Workload(args.slots_log2, args.batch_log2, args.lf)
        vals = []
        for _ in range(args.warmup):
            run_oracle_sample(args, args.cpu_sample_log2 - 2)
        for _ in range(args.steps):
            vals.append(run_oracle_sample(args, args.cpu_sample_log2))
        v = statistics.median(x["value"] for x in vals)
        cb = dict(vals[-1])
        cb["value"] = v
        n_s = 1 << args.cpu_sample_log2
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mops/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded splitmix64 keys)",
                "config": {"workload": f"map<u64,u64> {wl.slots} slots (capacity), timed on a bounded sample: "
                                       f"fill {n_s} keys, find {n_s // 4} hit + {n_s // 4} miss, erase {n_s // 4} "
                                       f"(the GPU arm's workload: {wl.name})",
                           "slots": wl.slots, "sample_keys": n_s, "batch": wl.batch, "load_factor": args.lf},
                "cpu_baseline": cb, "e2e": {"value": v, "unit": "Mops/s", "h2d_bytes_per_step": 0,
                                            "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_gpu(args, rank, world)
    if rank == 0:
        if not args.no_cpu and args.workload == "map_sweep":
            out["cpu_baseline"] = run_oracle_sample(args, args.cpu_sample_log2)
        shaped = args.bucket_bytes or args.lane_bytes or args.kpt or args.block or args.find_lane_bytes
        if world == 1 and args.workload == "map_sweep" and not args.no_extras and not shaped:
            out["workloads"] = run_extras(args)
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
