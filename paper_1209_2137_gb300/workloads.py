"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers; it holds none of the coding arithmetic,
so both the CUDA path's tests and the CPU oracle can take their inputs from it.

Randomness comes from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) in its
counter form: output i of a stream with seed s is mix(s + (i + 1) * gamma),
where mix is the published 64-bit finaliser.  Every workload uses a fixed seed
so a run is reproducible; the recipes stand in for the paper's synthetic
ClusterData / Uniform generators (whose definitions are not given in the
paper, Sec. 6.4) and for its TREC posting lists (Sec. 6.5), which are not
available here.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Seeds: a base plus the workload number, fixed so runs are comparable.
SEED_BASE = 20120910


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream `seed`."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _top_bits(z: np.ndarray, bits: int) -> np.ndarray:
    if bits == 0:
        return np.zeros(z.shape, dtype=np.uint64)
    return z >> np.uint64(64 - bits)


def uniform_u32(n: int, seed: int, bits: int = 32) -> np.ndarray:
    """n independent values uniform in [0, 2^bits)."""
    return _top_bits(splitmix64(seed, 0, n), bits).astype(np.uint32)


def _sorted_distinct(values: np.ndarray) -> np.ndarray:
    s = np.sort(values)
    if s.size == 0:
        return s
    keep = np.empty(s.size, dtype=bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def distinct_sorted(n: int, range_size: int, seed: int) -> np.ndarray:
    """n distinct values uniform in [0, range_size), sorted ascending.

    Draws n plus a margin of candidates, removes duplicates, and if more than
    n distinct values remain keeps the n whose keys from a second stream are
    smallest (a uniformly random n-subset of a uniform set)."""
    if n > range_size:
        raise ValueError("more distinct values than the range holds")
    margin = max(1024, n // 8)
    while True:
        z = splitmix64(seed, 0, n + margin)
        if range_size & (range_size - 1) == 0:
            cand = _top_bits(z, int(math.log2(range_size)))
        else:
            cand = z % np.uint64(range_size)
        u = _sorted_distinct(cand)
        if u.size >= n:
            break
        margin *= 4
    if u.size > n:
        keys = splitmix64(seed ^ 0x2545F4914F6CDD1D, 0, u.size)
        pick = np.sort(np.argpartition(keys, n - 1)[:n]) if n > 0 else np.zeros(0, dtype=np.int64)
        u = u[pick]
    return u.astype(np.uint32)


def uniform_sorted(n: int, range_bits: int, seed: int) -> np.ndarray:
    """Sorted distinct values uniform in [0, 2^range_bits) (Uniform model)."""
    return distinct_sorted(n, 1 << range_bits, seed)


def clustered_sorted(centres: int = 1024, per_centre: int = 65536, window_bits: int = 18,
                     range_bits: int = 29, seed: int = SEED_BASE + 20) -> np.ndarray:
    """ClusterData-like set: `centres` centres uniform in [0, 2^range_bits),
    each with `per_centre` points uniform in a 2^window_bits window around it,
    clamped to the range, then deduplicated and sorted."""
    c = _top_bits(splitmix64(seed, 0, centres), range_bits).astype(np.int64)
    z = splitmix64(seed ^ 0x5DEECE66D, 0, centres * per_centre)
    off = _top_bits(z, window_bits).astype(np.int64) - (1 << (window_bits - 1))
    pts = np.repeat(c, per_centre) + off
    np.clip(pts, 0, (1 << range_bits) - 1, out=pts)
    return _sorted_distinct(pts).astype(np.uint32)


def exception_heavy(n: int, seed: int = SEED_BASE + 3) -> np.ndarray:
    """Unsorted values, i.i.d. per position: with probability 0.9 geometric
    on {0, 1, ...} with success probability 1/9 (mean 8), otherwise uniform
    in [2^20, 2^28)."""
    sel = splitmix64(seed, 0, n)
    u = splitmix64(seed ^ 0x1234567, 0, n)
    big = splitmix64(seed ^ 0x7654321, 0, n)
    is_geo = (sel >> np.uint64(32)) % np.uint64(10) < np.uint64(9)
    # inverse CDF of the geometric law on (0, 1]
    unit = ((u >> np.uint64(11)).astype(np.float64) + 1.0) / float(1 << 53)
    geo = np.floor(np.log(unit) / math.log(8.0 / 9.0)).astype(np.int64)
    geo = np.minimum(geo, (1 << 20) - 1)
    wide = (1 << 20) + (big % np.uint64((1 << 28) - (1 << 20))).astype(np.int64)
    return np.where(is_geo, geo, wide).astype(np.uint32)


def random_small(n: int, seed: int, max_bits: int = 32) -> np.ndarray:
    """Values whose bit width varies per 128-value block (every width 0..max_bits
    occurs), for tests of the width-specialised paths."""
    z = splitmix64(seed, 0, n)
    widths = (splitmix64(seed ^ 0xABCDEF, 0, (n + 127) // 128) % np.uint64(max_bits + 1)).astype(np.int64)
    w = np.repeat(widths, 128)[:n]
    mask = np.where(w >= 32, np.uint64(0xFFFFFFFF), (np.uint64(1) << w.astype(np.uint64)) - np.uint64(1))
    return ((z >> np.uint64(32)) & mask).astype(np.uint32)


# -- named workloads ---------------------------------------------------------

def workload_sorted_small(seed: int = SEED_BASE + 1) -> np.ndarray:
    """65,536 distinct values uniform in [0, 2^22), sorted (deltas ~6 bits)."""
    return uniform_sorted(65536, 22, seed)


def workload_uniform_long(n: int = 1 << 26, seed: int = SEED_BASE + 2) -> np.ndarray:
    """2^26 distinct values uniform in [0, 2^29), sorted."""
    return uniform_sorted(n, 29, seed)


def workload_clustered_long(seed: int = SEED_BASE + 20) -> np.ndarray:
    """1,024 clusters of 65,536 points in 2^18 windows over [0, 2^29)."""
    return clustered_sorted(seed=seed)


def workload_exceptions(n: int = 1 << 26, seed: int = SEED_BASE + 3) -> np.ndarray:
    return exception_heavy(n, seed)


def posting_lists(nlists: int = 65536, total: int = 1 << 28, lo: int = 128, hi: int = 1 << 22,
                  alpha: float = 1.1, reading: str = "A", seed: int = SEED_BASE + 4):
    """Posting-list-like batch: list lengths Zipf(alpha) over [lo, hi].

    Reading "A": lengths drawn i.i.d. with P(L) ~ L^-alpha on [lo, hi]
    (inverse CDF of the continuous law, floored), then scaled by total/sum and
    clamped to [lo, hi].  Reading "B": rank-size L_r = hi * r^-alpha, clamped
    at lo.  Per list: beta uniform in {1..20} (the mean-delta bits), range
    R = min(L * 2^beta, 2^32), L distinct values uniform in [0, R), sorted;
    a coin picks the codec (True = SIMD-BP128 with stride-4 deltas, False =
    SIMD-FastPFOR with stride-1 deltas).

    Returns (lengths, offsets, values, bp128_mask)."""
    z = splitmix64(seed, 0, 3 * nlists)
    u = ((z[:nlists] >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)
    if reading == "A":
        a1 = 1.0 - alpha
        lo_p, hi_p = lo ** a1, hi ** a1
        L = np.floor((lo_p + u * (hi_p - lo_p)) ** (1.0 / a1))
        L = np.clip(np.floor(L * (total / L.sum())), lo, hi).astype(np.int64)
    elif reading == "B":
        r = np.arange(1, nlists + 1, dtype=np.float64)
        L = np.maximum(lo, np.round(hi * r ** (-alpha))).astype(np.int64)
    else:
        raise ValueError(reading)
    beta = 1 + (z[nlists:2 * nlists] % np.uint64(20)).astype(np.int64)
    bp = ((z[2 * nlists:] >> np.uint64(40)) & np.uint64(1)).astype(bool)
    offsets = np.zeros(nlists + 1, dtype=np.int64)
    np.cumsum(L, out=offsets[1:])
    values = np.empty(int(offsets[-1]), dtype=np.uint32)
    for i in range(nlists):
        n = int(L[i])
        R = min(n << int(beta[i]), 1 << 32)
        values[offsets[i]:offsets[i + 1]] = distinct_sorted(n, R, seed * 1000003 + i)
    return L, offsets, values, bp


def query_list(x: np.ndarray, nq: int, range_bits: int, seed: int, hit_frac: float = 0.5,
               distinct: bool = True) -> np.ndarray:
    """A sorted query list for intersecting with the sorted list x: about
    hit_frac * nq elements of x (positions drawn uniformly, with
    replacement) and the rest uniform in [0, 2^range_bits); sorted, and
    deduplicated if `distinct` (a posting list), else with its repeats."""
    nh = int(round(nq * hit_frac)) if x.size else 0
    z = splitmix64(seed, 0, nq)
    pos = (z[:nh] % np.uint64(max(1, x.size))).astype(np.int64)
    rest = _top_bits(z[nh:], range_bits).astype(np.uint32)
    q = np.concatenate([x[pos].astype(np.uint32), rest])
    return _sorted_distinct(q) if distinct else np.sort(q)


def workload_intersect(seed: int = SEED_BASE + 6):
    """The intersection workload: the 2^26-integer uniform list (values in
    [0, 2^29)) and a sorted distinct query list of about 2^22 integers, half
    of them drawn from the list (Sec. 7: lists of very different lengths)."""
    x = workload_uniform_long()
    return x, query_list(x, 1 << 22, 29, seed)
