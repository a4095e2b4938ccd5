"""Counter-based splitmix64 key streams (numpy, vectorised).

splitmix64 is Vigna's public-domain generator: the state advances by the
golden-ratio increment 0x9E3779B97F4A7C15 and each output is the state passed
through a xor-shift / multiply finaliser (shifts 30, 27, 31; multipliers
0xBF58476D1CE4E5B9 and 0x94D049BB133111EB).  Because the state after i steps is
just ``base + i * golden``, the i-th output can be computed directly, which
makes every stream random-access: ``stream_u64(stream, seed, start, n)`` is the
slice [start, start+n) of the sequence a sequential splitmix64 seeded with
``stream_base(stream, seed)`` would produce.

This module only draws inputs.  It holds none of the hash-container
arithmetic, so both the oracle and the GPU library may be fed from it.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 output finaliser applied elementwise to a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def mix_scalar(z: int) -> int:
    """Same finaliser on a Python int (mod 2^64)."""
    m = (1 << 64) - 1
    z &= m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def sequential(seed: int, n: int) -> list[int]:
    """First n outputs of a sequential splitmix64 seeded with ``seed``."""
    m = (1 << 64) - 1
    s = seed & m
    out = []
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & m
        out.append(mix_scalar(s))
    return out


def stream_base(stream: int, seed: int = 0) -> int:
    """Starting state of key stream ``stream`` under ``seed``."""
    return mix_scalar(((stream & 0xFFFFFFFF) << 32) ^ (seed & ((1 << 64) - 1)))


def stream_u64(stream: int, seed: int, start: int, n: int) -> np.ndarray:
    """Outputs start..start+n-1 of stream ``stream`` as uint64."""
    base = np.uint64(stream_base(stream, seed))
    i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix(base + i * GOLDEN)


def stream_at(stream: int, seed: int, idx: np.ndarray) -> np.ndarray:
    """Outputs at arbitrary indices ``idx`` (uint64/int64 array) of a stream."""
    base = np.uint64(stream_base(stream, seed))
    i = np.asarray(idx).astype(np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        return mix(base + i * GOLDEN)


def stream_u32(stream: int, seed: int, start: int, n: int) -> np.ndarray:
    """High 32 bits of the uint64 stream."""
    return (stream_u64(stream, seed, start, n) >> np.uint64(32)).astype(np.uint32)


def value_of(keys: np.ndarray) -> np.ndarray:
    """Map value drawn as splitmix64(key): the first output of a splitmix64
    seeded with the key's bit pattern."""
    k = np.asarray(keys).view(np.uint64) if np.asarray(keys).dtype.itemsize == 8 \
        else np.asarray(keys).astype(np.uint64)
    with np.errstate(over="ignore"):
        return mix(k + GOLDEN)


def uniform01(stream: int, seed: int, start: int, n: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the stream."""
    return (stream_u64(stream, seed, start, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def permutation(n: int, stream: int, seed: int = 0) -> np.ndarray:
    """A seeded permutation of range(n): indices ordered by their stream draw.

    Defined by a stable argsort so it is identical on every platform and numpy
    version (no dependence on numpy's own shuffling algorithms)."""
    r = stream_u64(stream, seed, 0, n)
    return np.argsort(r, kind="stable").astype(np.int64)


def affine_sample(n_pop: int, n: int, stream: int, seed: int = 0) -> np.ndarray:
    """n distinct indices in [0, n_pop), pseudo-randomly spread, without
    materialising a permutation of n_pop: j -> (a*j + c) mod n_pop with
    gcd(a, n_pop) = 1 is a bijection on [0, n_pop)."""
    assert 0 <= n <= n_pop
    a = (stream_base(stream, seed) % n_pop) | 1
    while np.gcd(a, n_pop) != 1:
        a += 2
    c = stream_base(stream + 1, seed) % n_pop
    j = np.arange(n, dtype=np.int64)
    # (a*j + c) mod n_pop without 64-bit overflow: split a into 2^20 chunks.
    a_hi, a_lo = a >> 20, a & ((1 << 20) - 1)
    t = (j * a_hi) % n_pop
    t = ((t << 20) % n_pop + (j * a_lo) % n_pop + c) % n_pop
    return t.astype(np.int64)
