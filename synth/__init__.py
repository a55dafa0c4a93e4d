"""Seeded synthetic workloads for the integer sort.

This module only draws inputs. It holds none of the sort's arithmetic, so the
oracle (``oracle/``) and the CUDA path (``paper_cs_0004013_gb300``) can both use
it without sharing any code with each other.

The paper's five contest data sets (Sec. 1.1, the key table) came from an
object file that is not available, so each is replaced by a seeded stand-in
with the property the paper lists for it:

=====  =====================  ==========================================
key    paper's description    stand-in here
=====  =====================  ==========================================
1      random / good balance  ``uniform31``
2      random / bad balance   ``skewed_chunks`` (64 chunks, max = 8x mean)
3      uniform / good         ``uniform31`` at 2^26, with payload
4      some clustering        ``gauss_mix`` (70% uniform, 30% clusters)
5      clustered              ``tight_clusters`` (8 clusters of 2^12)
=====  =====================  ==========================================

plus ``few_distinct`` (65,536 distinct values, heavy duplicates), the
segmented batch ``segment_sizes`` and the request stream ``serving_requests``.

Random numbers come from SplitMix64 (S. Vigna's public-domain generator, the
finaliser of Java's SplittableRandom): output i of stream s is
``mix(s + (i + 1) * 0x9E3779B97F4A7C15)``.  Being counter-based it vectorises
with numpy and gives the same numbers on x86 and Arm.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "CONFIG_SEED",
    "splitmix64",
    "uniform31",
    "skewed_chunk_sizes",
    "skewed_chunks",
    "few_distinct",
    "gauss_mix",
    "tight_clusters",
    "segment_sizes",
    "segmented_batch",
    "serving_requests",
    "config_keys",
    "DISTRIBUTIONS",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

#: base seed of workload ``c`` is ``CONFIG_SEED + c``; sub-streams add a salt.
CONFIG_SEED = 0x5EED0000


def _stream_seed(seed: int, salt: int = 0) -> np.uint64:
    # Distinct sub-streams: salt the seed through one SplitMix64 step so that
    # seeds s and s+1 do not produce overlapping counter ranges.
    return np.uint64(int(splitmix64(seed ^ (salt * 0xD1B54A32D192ED03 & _MASK64), 1)[0]))


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+n-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK64) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _u01(seed: int, n: int, salt: int) -> np.ndarray:
    """Uniform doubles in (0, 1): 53 high bits, offset by half an ulp."""
    z = splitmix64(int(_stream_seed(seed, salt)), n)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / (1 << 53))


def _below(seed: int, n: int, bound: int, salt: int) -> np.ndarray:
    """Integers in [0, bound): the high bits of a 64-bit draw times bound
    (Lemire's multiply-shift; bias < bound / 2^64, negligible here)."""
    z = splitmix64(int(_stream_seed(seed, salt)), n)
    hi = z >> np.uint64(32)
    lo = z & np.uint64(0xFFFFFFFF)
    b = np.uint64(bound)
    # (z * bound) >> 64 computed in two 32-bit halves to stay inside uint64.
    with np.errstate(over="ignore"):
        t = (lo * b) >> np.uint64(32)
        return ((hi * b + t) >> np.uint64(32)).astype(np.int64)


def uniform31(n: int, seed: int) -> np.ndarray:
    """n keys uniform in [0, 2^31 - 1] (the top 31 bits of each draw)."""
    return (splitmix64(seed, n) >> np.uint64(33)).astype(np.uint32)


def skewed_chunk_sizes(n: int, chunks: int, seed: int, max_over_mean: int = 8) -> np.ndarray:
    """Sizes of ``chunks`` source chunks summing to n, the largest being
    ``max_over_mean`` times the mean: one chunk takes n*max/chunks, the others
    share the rest with lognormal weights (sigma 1), each capped below that
    maximum, rounded by largest remainder."""
    mean = n / chunks
    big = int(round(max_over_mean * mean))
    rest = n - big
    z = _u01(seed, 2 * (chunks - 1), salt=11)
    g = np.sqrt(-2.0 * np.log(z[0::2])) * np.cos(2.0 * math.pi * z[1::2])
    w = np.exp(g)
    w = w / w.sum() * rest
    w = np.minimum(w, big - 1)
    w = w / w.sum() * rest
    base = np.floor(w).astype(np.int64)
    short = rest - int(base.sum())
    order = np.argsort(-(w - base), kind="stable")
    base[order[:short]] += 1
    sizes = np.concatenate([[big], base])
    # place the big chunk at a seeded position so it is not always first
    pos = int(_below(seed, 1, chunks, salt=12)[0])
    sizes = np.roll(sizes, pos)
    assert int(sizes.sum()) == n
    return sizes


def skewed_chunks(n: int, seed: int, chunks: int = 64) -> np.ndarray:
    """Key 2 stand-in: 64 chunks of skewed sizes (largest 8x the mean), each
    drawn from its own uniform 31-bit stream, concatenated in chunk order."""
    sizes = skewed_chunk_sizes(n, chunks, seed)
    parts = [uniform31(int(s), int(_stream_seed(seed, 100 + c))) for c, s in enumerate(sizes)]
    return np.concatenate(parts).astype(np.uint32)


def few_distinct(n: int, seed: int, distinct: int = 65536) -> np.ndarray:
    """Keys drawn uniformly from ``distinct`` distinct uniform 31-bit values."""
    vals = np.unique(uniform31(2 * distinct + 1024, int(_stream_seed(seed, 21))))
    # take the first `distinct` of a seeded shuffle of the unique values
    perm = np.argsort(splitmix64(int(_stream_seed(seed, 22)), vals.size), kind="stable")
    vals = vals[perm[:distinct]]
    assert vals.size == distinct
    return vals[_below(seed, n, distinct, salt=23)].astype(np.uint32)


def gauss_mix(n: int, seed: int, clusters: int = 16, sigma: float = float(1 << 20),
              frac: float = 0.3) -> np.ndarray:
    """Key 4 stand-in: each key is, with probability ``frac``, drawn from one
    of 16 Gaussian clusters (sigma 2^20, uniform 31-bit centres; Box-Muller in
    double, rounded to nearest, clamped to [0, 2^31-1]); otherwise uniform
    31-bit."""
    u = uniform31(n, int(_stream_seed(seed, 31))).astype(np.int64)
    pick = _u01(seed, n, salt=32) < frac
    centres = uniform31(clusters, int(_stream_seed(seed, 33))).astype(np.float64)
    which = _below(seed, n, clusters, salt=34)
    z1 = _u01(seed, n, salt=35)
    z2 = _u01(seed, n, salt=36)
    g = np.sqrt(-2.0 * np.log(z1)) * np.cos(2.0 * math.pi * z2)
    c = np.rint(centres[which] + sigma * g)
    c = np.clip(c, 0, (1 << 31) - 1).astype(np.int64)
    return np.where(pick, c, u).astype(np.uint32)


def tight_clusters(n: int, seed: int, clusters: int = 8, width: int = 4096) -> np.ndarray:
    """Key 5 stand-in: every key is base_c + U[0, width-1], with the cluster c
    uniform over ``clusters`` bases uniform in [0, 2^31 - width]."""
    bases = _below(seed, clusters, (1 << 31) - width + 1, salt=41)
    which = _below(seed, n, clusters, salt=42)
    off = _below(seed, n, width, salt=43)
    return (bases[which] + off).astype(np.uint32)


DISTRIBUTIONS = {
    "uniform": lambda n, seed: uniform31(n, seed),
    "skewed_chunks": lambda n, seed: skewed_chunks(n, seed),
    "few_distinct": lambda n, seed: few_distinct(n, seed),
    "gauss_mix": lambda n, seed: gauss_mix(n, seed),
    "tight_clusters": lambda n, seed: tight_clusters(n, seed),
}


def config_keys(config: int, n: int | None = None, dist: str = "uniform") -> np.ndarray:
    """Keys of workload 1 (2^20 uniform), 2 (2^26 uniform) or 3 (2^26, one of
    the four distributions), at the stated size unless ``n`` is given."""
    if n is None:
        n = 1 << 20 if config == 1 else 1 << 26
    return DISTRIBUTIONS[dist](n, CONFIG_SEED + config)


def segment_sizes(seed: int, max_segments: int = 4096, lo: int = 1 << 10, hi: int = 1 << 20,
                  cap: int = 1 << 28) -> np.ndarray:
    """Log-uniform segment sizes floor(exp(U(ln lo, ln hi))), drawn in order,
    at most ``max_segments`` of them, stopping before the first one that would
    push the total above ``cap``."""
    u = _u01(seed, max_segments, salt=51)
    s = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    s = np.clip(s, lo, hi)
    tot = np.cumsum(s)
    keep = int(np.searchsorted(tot, cap, side="right"))
    return s[:keep]


def segmented_batch(seed: int, **kw) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(keys, vals, seg_offsets): concatenated uniform 31-bit keys of the
    segments of ``segment_sizes``; vals = global index (checks stability)."""
    sizes = segment_sizes(seed, **kw)
    offs = np.zeros(sizes.size + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(sizes)
    n = int(offs[-1])
    keys = uniform31(n, int(_stream_seed(seed, 52)))
    vals = np.arange(n, dtype=np.uint32)
    return keys, vals, offs


def serving_requests(count: int, seed: int, rate_per_s: float, lo: int = 1 << 16,
                     hi: int = 1 << 26) -> list[dict]:
    """A Poisson request stream: exponential inter-arrival gaps at
    ``rate_per_s``, log-uniform sizes in [lo, hi], and each request keys-only
    (like workload 1) or key+payload (like workload 2) with probability 1/2.
    Each request carries its own key seed."""
    gaps = -np.log(_u01(seed, count, salt=61)) / rate_per_s
    arrive = np.cumsum(gaps) - gaps[0]
    u = _u01(seed, count, salt=62)
    sizes = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    pairs = _u01(seed, count, salt=63) < 0.5
    out = []
    for i in range(count):
        out.append({"id": i, "arrival_s": float(arrive[i]), "n": int(min(max(sizes[i], lo), hi)),
                    "pairs": bool(pairs[i]), "seed": int(_stream_seed(seed, 1000 + i))})
    return out
