"""Random-read rate of the current GPU: the ceiling of probe-bound operations.

    python -m paper_1908_05936_gb300.probe [--gib 2] [--reads-log2 26] [--reps 5]
    python -m paper_1908_05936_gb300.probe --sweep
    python -m paper_1908_05936_gb300.probe --same-line [--gib 4]

Times hc_measure_random_reads (32-byte reads at random 32-byte-aligned
offsets of a device buffer larger than L2) and prints one JSON line; with
--sweep, one line per buffer size from 8 MiB (inside L2) to 16 GiB; with
--same-line, hc_measure_line_reads: one random line per key read once, twice
together, or twice with the second read after the first (three lines).
"""
from __future__ import annotations

import argparse
import ctypes
import json


def measure(gib: float = 2.0, reads_log2: int = 26, reps: int = 5) -> dict:
    import torch

    from . import _lib as L
    from . import build
    build.build()
    buf = torch.empty(int(gib * (1 << 30)), dtype=torch.uint8, device="cuda")
    ms = ctypes.c_float()
    n = 1 << reads_log2
    L.check(L.load().hc_measure_random_reads(buf.data_ptr(), buf.numel(), n, reps, ctypes.byref(ms),
                                             torch.cuda.current_stream().cuda_stream))
    rate = n / (ms.value * 1e-3)
    return {"reads": n, "buffer_bytes": buf.numel(), "ms_per_launch": round(ms.value, 4),
            "g_reads_per_s": round(rate / 1e9, 2), "sector_gbs": round(rate * 32 / 1e9, 1),
            "line_gbs": round(rate * 128 / 1e9, 1)}


def same_line(gib: float = 4.0, keys_log2: int = 26, reps: int = 5) -> list[dict]:
    import torch

    from . import _lib as L
    from . import build
    build.build()
    buf = torch.zeros(int(gib * (1 << 30)), dtype=torch.uint8, device="cuda")
    n = 1 << keys_log2
    out = []
    for reads, dep, name in ((1, 0, "one read"), (2, 0, "two reads of the line, together"),
                             (2, 1, "two reads of the line, the second after the first")):
        ms = ctypes.c_float()
        L.check(L.load().hc_measure_line_reads(buf.data_ptr(), buf.numel(), n, reads, dep, reps, ctypes.byref(ms),
                                               torch.cuda.current_stream().cuda_stream))
        out.append({"mode": name, "keys": n, "buffer_bytes": buf.numel(), "ms_per_launch": round(ms.value, 4),
                    "g_keys_per_s": round(n / (ms.value * 1e-3) / 1e9, 2),
                    "g_requests_per_s": round(reads * n / (ms.value * 1e-3) / 1e9, 2)})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gib", type=float, default=None, help="buffer GiB (2 for reads, 4 for --same-line)")
    ap.add_argument("--reads-log2", type=int, default=26)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--same-line", action="store_true")
    a = ap.parse_args()
    if a.same_line:
        for row in same_line(a.gib or 4.0, a.reads_log2, a.reps):
            print(json.dumps(row))
        return
    if a.sweep:
        import torch
        for mib in (8, 32, 64, 96, 128, 256, 512, 1024, 2048, 4096, 8192, 16384):
            print(json.dumps(measure(mib / 1024, a.reads_log2, a.reps)), flush=True)
            torch.cuda.empty_cache()
        return
    print(json.dumps(measure(a.gib or 2.0, a.reads_log2, a.reps)))


if __name__ == "__main__":
    main()
