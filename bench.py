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
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample-log2", type=int, default=22)
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

    bb = args.bucket_bytes or 32
    t = Table(L.MAP_U64_U64, wl.slots, bucket_bytes=bb)
    for op in (0, 1, 2):
        t.set_launch(op, lane_bytes=args.lane_bytes, keys_per_group=args.kpt, block=args.block)
    stream = torch.cuda.current_stream()
    calls = []   # (name, n, start_event, end_event)

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
            t.insert(d_fill[off:off + n], d_vals[off:off + n], status=st_buf[:n])
            b = ev()
            rec.append(("insert", n, a, b))
        a = ev()
        t.find(d_hit, found=found, vals_out=vout)
        b = ev()
        rec.append(("find_hit", B, a, b))
        a = ev()
        t.find(d_miss, found=found, vals_out=vout)
        b = ev()
        rec.append(("find_miss", B, a, b))
        a = ev()
        t.erase(d_er, status=st_buf)
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
    if world > 1:
        tt = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        elapsed_ms = float(tt.item())

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

    ops = wl.ops_per_step() * args.steps * world
    value = ops / (elapsed_ms * 1e-3) / 1e6

    # roofline of the dominant kernel (largest share of the timed region)
    kinds = {"insert": "insert", "find_hit": "find", "find_miss": "find", "erase": "erase"}
    dom = max((k for k in per if k in kinds), key=lambda k: summary[k]["ms_total"])
    dom_n = sum(x[0] for x in per[dom]) / len(per[dom])
    dom_ms = summary[dom]["ms_total"] / len(per[dom])
    achieved = BYTES_PER_OP[kinds[dom]] * dom_n / (dom_ms * 1e-3) / 1e9
    peak, peak_src = hbm_peak()

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mops/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded splitmix64 keys)",
        "config": {"workload": wl.name, "slots": wl.slots, "batch": B, "load_factor": args.lf,
                   "bucket_bytes": bb, "launch": t.get_launch(1), "l2": "inputs larger than L2 (4 GiB table)",
                   "parallelism": f"replicas{world}"},
        "ops": {k: ({kk: round(vv, 4) if isinstance(vv, float) else vv for kk, vv in v.items()}
                    if isinstance(v, dict) else v) for k, v in summary.items()},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                     "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": None, "bytes_per_op": BYTES_PER_OP[kinds[dom]]},
        "clocks": clk,
        "gpu_launches": len(calls) * world,
        "check": {"size_after_step": size_after, "expected": expected_size},
    }
    if not args.no_e2e:
        out["e2e"] = run_e2e(t, wl, fill, vals, hit, miss, er, stream)
    t.close()
    return out


def run_e2e(t, wl, fill, vals, hit, miss, er, stream):
    """Same step through the C ABI's host-buffer calls: pinned host arrays in,
    host results out, every copy inside the timed region."""
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
            "d2h_bytes_per_step": int(d2h), "ms_per_step": round(dt * 1e3, 2)}


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


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
    t0 = time.perf_counter()
    t.insert(fill, vals)
    t.find(hit)
    t.find(miss)
    t.erase(er)
    dt = time.perf_counter() - t0
    t.close()
    ops = n + 3 * q
    return {"value": round(ops / dt / 1e6, 3), "unit": "Mops/s", "cores": 1, "kind": "oracle",
            "sample": f"fill {n} keys, find {q} hit + {q} miss, erase {q} (single-threaded C chained table)",
            "seconds": round(dt, 2), "host_cores_available": os.cpu_count()}


def main():
    args = parse()
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
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mops/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded splitmix64 keys)",
                "config": {"workload": wl.name, "slots": wl.slots, "batch": wl.batch, "load_factor": args.lf},
                "cpu_baseline": cb, "e2e": {"value": v, "unit": "Mops/s", "h2d_bytes_per_step": 0,
                                            "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_gpu(args, rank, world)
    if rank == 0:
        if not args.no_cpu:
            out["cpu_baseline"] = run_oracle_sample(args, args.cpu_sample_log2)
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
