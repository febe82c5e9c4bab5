"""Seeded synthetic workload generators.

This module only draws inputs: keys, bucket sizes and request streams.  It
holds none of the peeling or hashing arithmetic, and both the CUDA library's
tests and the CPU oracle take their inputs from here.

Keys stand in for the paper's string data sets (sec. 5 "Datasets": the keys
are hashed first, and random keys gave the same results).  Keys are SplitMix64
streams (Steele, Lea, Flood, OOPSLA 2014): key i of stream ``seed`` is the
(i+1)-th output of a SplitMix64 generator whose state starts at ``seed``.
Every output is a bijective image of a distinct state, so a stream has no
duplicate keys.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _splitmix_out(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_stream(seed: int, n: int, start: int = 0,
                      chunk: int = 1 << 24) -> np.ndarray:
    """uint64[n]: outputs start+1 .. start+n of SplitMix64 seeded with ``seed``."""
    out = np.empty(n, dtype=np.uint64)
    s = np.uint64(seed & (2**64 - 1))
    with np.errstate(over="ignore"):
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            i = np.arange(start + a + 1, start + b + 1, dtype=np.uint64)
            out[a:b] = _splitmix_out(s + i * _GOLDEN)
    return out


def keys(n: int, seed: int = 1) -> np.ndarray:
    """The key set of a single-graph workload: uint64[n], distinct."""
    return splitmix64_stream(seed, n)


def _signed(x: int) -> int:
    x &= 2**64 - 1
    return x - 2**64 if x >= 2**63 else x


def keys_torch(n: int, seed: int = 1, device="cuda", chunk: int = 1 << 27):
    """keys(n, seed) generated with torch int64 operations on ``device``
    (two's-complement products wrap modulo 2^64; right shifts are made
    logical with a mask), in chunks: the same values, without the host
    array.  Returns a torch.int64 tensor holding the uint64 bit patterns."""
    import torch

    out = torch.empty(n, dtype=torch.int64, device=device)
    golden, m1, m2 = _signed(0x9E3779B97F4A7C15), _signed(0xBF58476D1CE4E5B9), \
        _signed(0x94D049BB133111EB)
    s = _signed(seed)

    def lsr(z, k):
        return (z >> k) & ((1 << (64 - k)) - 1)

    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        z = torch.arange(a + 1, b + 1, dtype=torch.int64, device=device) * golden + s
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        out[a:b] = z ^ lsr(z, 31)
    return out


def uniforms53(seed: int, n: int) -> np.ndarray:
    """float64[n] in [0, 1): top 53 bits of a SplitMix64 stream."""
    return (splitmix64_stream(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def lognormal_bucket_sizes(B: int = 65536, median: int = 2000, sigma: float = 0.92,
                           lo: int = 64, hi: int = 65536, seed: int = 3) -> np.ndarray:
    """Bucket sizes for the batched workload: clip(round(exp(ln median + sigma Z)),
    lo, hi), Z standard normal by Box-Muller over a SplitMix64 uniform stream."""
    u = uniforms53(seed, 2 * ((B + 1) // 2))
    u1 = np.maximum(u[0::2], 2.0 ** -53)
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([rad * np.cos(2 * math.pi * u2), rad * np.sin(2 * math.pi * u2)])
    z = z.reshape(2, -1).T.reshape(-1)[:B]
    s = np.rint(np.exp(math.log(median) + sigma * z))
    return np.clip(s, lo, hi).astype(np.int64)


def bucketed_keys(sizes: np.ndarray, seed: int = 2):
    """(keys uint64[total], offsets uint64[B+1]): one SplitMix64 stream cut into
    consecutive buckets of the given sizes."""
    off = np.zeros(len(sizes) + 1, dtype=np.uint64)
    off[1:] = np.cumsum(sizes, dtype=np.uint64)
    return splitmix64_stream(seed, int(off[-1])), off


def request_stream(num: int, rate_per_s: float, seed: int = 4, lo_exp: float = 3.0,
                   hi_exp: float = 7.0):
    """Serving workload: (arrival times s, key-set sizes, key seeds).  Sizes are
    floor(10^(lo + (hi-lo) U)); inter-arrival gaps are exponential (Poisson)."""
    u = uniforms53(seed, 2 * num)
    sizes = np.floor(10.0 ** (lo_exp + (hi_exp - lo_exp) * u[0::2])).astype(np.int64)
    gaps = -np.log(np.maximum(1.0 - u[1::2], 2.0 ** -53)) / rate_per_s
    arrivals = np.cumsum(gaps)
    seeds = 1000 + np.arange(num, dtype=np.int64)
    return arrivals, sizes, seeds
