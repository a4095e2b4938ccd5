"""Random-read rate of the current GPU: the ceiling of probe-bound operations.

    python -m paper_1908_05936_gb300.probe [--gib 2] [--reads-log2 26] [--reps 5]
    python -m paper_1908_05936_gb300.probe --sweep

Times hc_measure_random_reads (32-byte reads at random 32-byte-aligned
offsets of a device buffer larger than L2) and prints one JSON line; with
--sweep, one line per buffer size from 8 MiB (inside L2) to 16 GiB.
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gib", type=float, default=2.0)
    ap.add_argument("--reads-log2", type=int, default=26)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--sweep", action="store_true")
    a = ap.parse_args()
    if a.sweep:
        import torch
        for mib in (8, 32, 64, 96, 128, 256, 512, 1024, 2048, 4096, 8192, 16384):
            print(json.dumps(measure(mib / 1024, a.reads_log2, a.reps)), flush=True)
            torch.cuda.empty_cache()
        return
    print(json.dumps(measure(a.gib, a.reads_log2, a.reps)))


if __name__ == "__main__":
    main()
