"""Seeded synthetic workloads shaped like the hash-container workloads.

Every array here is drawn from counter-based splitmix64 streams
(``workloads.splitmix``), so a workload is reproducible from its
(stream, seed) pairs alone, on any machine.  Stream ids by role:

  1, 2       set<u32> workload: inserted keys / fresh query keys
  3, 4       map<u64,u64> sweep: inserted keys / fresh (missing) query keys
  10..19     permutations and samples
  1000 + t   multi-table workload, table t (inserts), 5000 + t (fresh finds)
  3000..     served workload (arrivals, sizes, ops, ranks)
  40..42     batches with repeated keys: the key domain, draws, op kinds
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import splitmix as sm

# ---------------------------------------------------------------------------
# set<uint32>, 2^21 slots: insert 1M, find 1M (half present), erase 500k
# ---------------------------------------------------------------------------


@dataclass
class SetU32Workload:
    slots: int
    insert_keys: np.ndarray   # uint32[n_insert]
    find_keys: np.ndarray     # uint32[n_find]
    erase_keys: np.ndarray    # uint32[n_erase]


def set_u32_workload(n_insert: int = 1_000_000, n_find: int = 1_000_000,
                     n_erase: int = 500_000, slots: int = 1 << 21,
                     seed: int = 0) -> SetU32Workload:
    """Uniform u32 keys (stream 1); queries are half a seeded sample of the
    inserted keys and half fresh keys (stream 2), shuffled together; erases are
    a seeded sample, without replacement, of the insert positions."""
    ins = sm.stream_u32(1, seed, 0, n_insert)
    n_hit = n_find // 2
    hit_pos = sm.permutation(n_insert, 10, seed)[:n_hit]
    fresh = sm.stream_u32(2, seed, 0, n_find - n_hit)
    q = np.concatenate([ins[hit_pos], fresh])
    q = q[sm.permutation(n_find, 11, seed)]
    er_pos = sm.permutation(n_insert, 12, seed)[:n_erase]
    return SetU32Workload(slots, ins, q, ins[er_pos])


# ---------------------------------------------------------------------------
# map<uint64,uint64>, 2^28 slots: fill to a load factor, find hit / miss, erase
# ---------------------------------------------------------------------------

MAP_SWEEP_SLOTS = 1 << 28
MAP_SWEEP_LOAD_FACTORS = (0.5, 0.7, 0.8, 0.9)
MAP_SWEEP_BATCHES = tuple(1 << e for e in (16, 18, 20, 22, 24, 26))


def fill_count(slots: int, load_factor: float) -> int:
    """Keys inserted to reach a load factor (floor, as in 0.8 * 2^28)."""
    return int(math.floor(load_factor * slots))


def map_fill_keys(start: int, n: int, seed: int = 0) -> np.ndarray:
    """Inserted keys [start, start+n) of the sweep (stream 3)."""
    return sm.stream_u64(3, seed, start, n)


def map_hit_keys(n_inserted: int, n: int, seed: int = 0, salt: int = 0) -> np.ndarray:
    """n distinct inserted keys, spread over the whole inserted range."""
    idx = sm.affine_sample(n_inserted, n, 14 + 2 * salt, seed)
    return sm.stream_at(3, seed, idx)


def map_miss_keys(n: int, seed: int = 0, start: int = 0) -> np.ndarray:
    """Fresh keys (stream 4): absent unless a 2^-64-per-pair collision hits."""
    return sm.stream_u64(4, seed, start, n)


def repeated_keys(n: int, n_distinct: int, seed: int = 0) -> np.ndarray:
    """n draws, uniform with replacement, from n_distinct fresh uint64 keys
    (stream 40 holds the domain, stream 41 the draws): each key appears
    n / n_distinct times on average, in scattered positions."""
    u = sm.uniform01(41, seed, 0, n)
    idx = np.minimum((u * n_distinct).astype(np.int64), n_distinct - 1)
    return sm.stream_at(40, seed, idx)


def mixed_ops(n: int, mix=(0.5, 0.3, 0.2), seed: int = 0) -> np.ndarray:
    """Op kinds of a mixed batch (0 insert, 1 find, 2 erase) drawn
    independently per position with probabilities `mix` (stream 42)."""
    u = sm.uniform01(42, seed, 0, n)
    return np.where(u < mix[0], 0, np.where(u < mix[0] + mix[1], 1, 2)).astype(np.uint8)


# ---------------------------------------------------------------------------
# Multi-table workload: 1024 set<u64>, capacities log-uniform in 2^10..2^22
# ---------------------------------------------------------------------------


@dataclass
class TableOps:
    slots: int
    insert_keys: np.ndarray
    find_keys: np.ndarray
    erase_keys: np.ndarray


def multi_table_slots(n_tables: int = 1024, lo_exp: float = 10, hi_exp: float = 22,
                      multiple: int = 16, seed: int = 0) -> np.ndarray:
    """Capacities round(2^U(lo,hi)) rounded up to a multiple of ``multiple``."""
    u = sm.uniform01(20, seed, 0, n_tables)
    s = np.round(np.exp2(lo_exp + (hi_exp - lo_exp) * u)).astype(np.int64)
    return ((s + multiple - 1) // multiple) * multiple


def multi_table_ops(slots: int, t: int, seed: int = 0, ops_fraction: float = 0.5,
                    mix=(0.6, 0.3, 0.1)) -> TableOps:
    """Ops for table t: 0.5*slots ops split 60/30/10 into insert (uniform u64,
    stream 1000+t), find (half this batch's inserts, half fresh from stream
    5000+t) and erase (a sample of this batch's inserts)."""
    n = int(round(ops_fraction * slots))
    n_ins = int(round(mix[0] * n))
    n_find = int(round(mix[1] * n))
    n_er = max(0, n - n_ins - n_find)
    ins = sm.stream_u64(1000 + t, seed, 0, n_ins)
    n_hit = n_find // 2
    hit = ins[sm.affine_sample(n_ins, min(n_hit, n_ins), 30, seed + t)] if n_ins else ins[:0]
    fresh = sm.stream_u64(5000 + t, seed, 0, n_find - len(hit))
    q = np.concatenate([hit, fresh])
    if len(q):
        q = q[sm.permutation(len(q), 31, seed + t)]
    er = ins[sm.affine_sample(n_ins, min(n_er, n_ins), 32, seed + t)] if n_ins else ins[:0]
    return TableOps(int(slots), ins, q, er)


# ---------------------------------------------------------------------------
# Served workload: Poisson arrivals of insert/find/erase requests on resident
# map<u64,u64> tables, sizes log-uniform in [1, 2^20], Zipf(1.1) keys
# ---------------------------------------------------------------------------


@dataclass
class Request:
    rid: int
    table: int
    op: int            # 0 insert, 1 find, 2 erase
    n: int
    arrival: float     # seconds from the start
    key_stream: int    # keys = zipf_keys(table, key_stream, n)


def zipf_cdf(n_ranks: int, s: float = 1.1) -> np.ndarray:
    """CDF of a Zipf(s) law over ranks 1..n_ranks (float64)."""
    w = np.arange(1, n_ranks + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_keys(table: int, stream: int, n: int, cdf: np.ndarray, seed: int = 0) -> np.ndarray:
    """n keys of one table: Zipf ranks by inverse CDF, mapped to uint64 keys
    through splitmix64(rank ^ table << 48) so hot keys are scattered."""
    u = sm.uniform01(stream, seed, 0, n)
    rank = np.searchsorted(cdf, u, side="right").astype(np.uint64)
    return sm.mix(rank ^ (np.uint64(table) << np.uint64(48)))


def served_requests(n_requests: int, n_tables: int, rate_per_s: float, seed: int = 0,
                    mix=(0.4, 0.5, 0.1), max_log2: int = 20) -> list[Request]:
    """Poisson arrivals (exponential gaps at `rate_per_s`), uniform table,
    op drawn from `mix`, size floor(2^U(0, max_log2))."""
    u = sm.uniform01(3000, seed, 0, 4 * n_requests).reshape(4, n_requests)
    gaps = -np.log(np.maximum(u[0], 1e-300)) / rate_per_s
    arrival = np.cumsum(gaps) - gaps[0]
    table = np.minimum((u[1] * n_tables).astype(np.int64), n_tables - 1)
    cm = np.cumsum(mix)
    op = np.searchsorted(cm / cm[-1], u[2], side="right")
    size = np.maximum(1, np.floor(np.exp2(u[3] * max_log2)).astype(np.int64))
    return [Request(i, int(table[i]), int(op[i]), int(size[i]), float(arrival[i]), 4000 + i)
            for i in range(n_requests)]
