"""Oracle for the integer sort: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library (``paper_cs_0004013_gb300``)
never imports it and shares no code with it; when the CUDA library is missing
the library fails instead of falling back to anything here.

What the sort computes has a plain definition, so the oracle is that
definition written out with numpy, with no blocking, fusion or reordering:

* the sorted output is the keys in ascending unsigned order (Sec. 1.1: cell 0
  holds the lowest values, cell 63 the highest);
* with a payload, equal keys keep their input order: the method is a radix
  sort in which the order reached on the lower digits survives the sorting by
  the higher ones (Sec. 3.3.1), and the order inside a bucket must survive
  distribution (Sec. 5);
* key words of other kinds (``order_perm``): two's-complement signed, and
  IEEE-754 binary32 in the standard's totalOrder (IEEE 754-2008 Sec. 5.10);
* the output is split into ``P`` (= 64) equal contiguous partitions, the lower
  partitions taking the extra element when P does not divide n (Sec. 1.1, and
  the rule in footnote 7 of Sec. 3.4.2 that the lower cell gets the odd datum).

The intermediate steps of the radix distribution are also given here, each as
its definition, so that every kernel step can be checked on its own:

* ``digit_histograms``: the count loop of the bucketing phase (Sec. 3.2) for
  every digit at once;
* ``digit_bases``: the cumulative bucket totals of Sec. 3.2, exclusive, i.e.
  the number of keys whose digit is smaller (Sec. 4.4 orders it as
  cumulative-then-sum, which gives the same numbers);
* ``distribute``: one stable distribution by a digit, the partial sort of
  Sec. 3.2 (grouped by bucket, buckets ascending) that keeps the earlier order
  (Sec. 3.3.1);
* ``skippable_digits``: a digit on which every key agrees moves nothing; the
  paper's 30-bit observation (Sec. 4.5) is the case of the top digit.

* ``choose_plan``: the selection of Sec. 4.2.1 (a sample of evenly spaced
  elements, each cell's overlap with its left neighbour's maximum, the 65 %
  rule, more than two problem cells abandoning the bucketing algorithm),
  written for the output partitions after bucketing by the top bits.

Pins against things other than itself live in ``tests/test_oracle.py``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "KINDS",
    "order_perm",
    "sort_keys",
    "sort_pairs",
    "partition_offsets",
    "sort_segmented",
    "merge",
    "digit_plan",
    "digit_of",
    "digit_histograms",
    "digit_bases",
    "skippable_digits",
    "distribute",
    "lsd_sort",
    "msd_buckets",
    "ordered_words",
    "selection_sample",
    "choose_plan",
]


def _u32(a) -> np.ndarray:
    a = np.asarray(a)
    if a.dtype != np.uint32:
        a = a.astype(np.uint32)
    return a


KINDS = ("u32", "i32", "f32", "u64", "i64", "f64")


def _words(keys, kind: str) -> np.ndarray:
    if kind.endswith("64"):
        a = np.asarray(keys)
        return a if a.dtype == np.uint64 else a.astype(np.uint64)
    return _u32(keys)


def order_perm(keys, kind: str = "u32") -> np.ndarray:
    """The stable permutation that puts key words (32- or 64-bit) in
    ascending order of their ``kind``:

    * ``u32`` / ``u64``: unsigned integers (Sec. 1.1);
    * ``i32`` / ``i64``: two's-complement signed integers;
    * ``f32`` / ``f64``: IEEE-754 binary32 / binary64 values in the
      totalOrder of IEEE 754-2008 Sec. 5.10: a value with the sign bit set
      comes before one without (so -NaN < -inf < -0 < +0 < +inf < +NaN);
      among negative ones the larger magnitude (the bits below the sign read
      as an integer, NaN payloads included) comes first, among non-negative
      ones the smaller.
    """
    w = _words(keys, kind)
    if kind in ("u32", "u64"):
        return np.argsort(w, kind="stable")
    if kind == "i32":
        return np.argsort(w.view(np.int32), kind="stable")
    if kind == "i64":
        return np.argsort(w.view(np.int64), kind="stable")
    if kind in ("f32", "f64"):
        bits = 32 if kind == "f32" else 64
        top = w.dtype.type(bits - 1)
        negative = (w >> top).astype(bool)
        magnitude = (w & w.dtype.type((1 << (bits - 1)) - 1)).astype(np.int64)
        within = np.where(negative, -magnitude, magnitude)
        sign_class = np.where(negative, 0, 1)
        return np.lexsort((within, sign_class))  # the last key is the primary one; lexsort is stable
    raise ValueError(f"unknown key kind {kind!r}")


def sort_keys(keys, kind: str = "u32") -> np.ndarray:
    """Keys in ascending order of their kind (unsigned 32-bit by default,
    Sec. 1.1); the words themselves are returned unchanged."""
    if kind == "u32":
        return np.sort(_u32(keys), kind="stable")
    w = _words(keys, kind)
    return w[order_perm(w, kind)]


def sort_pairs(keys, vals, kind: str = "u32") -> tuple[np.ndarray, np.ndarray]:
    """(key, value) pairs ordered by key alone; equal keys keep input order
    (Sec. 3.3.1, Sec. 5)."""
    keys = _words(keys, kind)
    vals = np.asarray(vals)
    if vals.dtype != np.uint64:  # payloads of 32 bits, or 64 bits carried as they are
        vals = _u32(vals)
    if keys.shape != vals.shape:
        raise ValueError("keys and vals differ in length")
    perm = order_perm(keys, kind)
    return keys[perm], vals[perm]


def merge(a, b, va=None, vb=None, kind: str = "u32"):
    """The stable merge of two sorted runs: the run a followed by the run b,
    sorted stably by key (so an element of a precedes an equal one of b).
    Returns (keys, vals or None)."""
    keys = np.concatenate([_words(a, kind), _words(b, kind)])
    if va is None:
        return keys[order_perm(keys, kind)], None
    vals = np.concatenate([_u32(va), _u32(vb)])
    perm = order_perm(keys, kind)
    return keys[perm], vals[perm]


def partition_offsets(n: int, num_parts: int = 64) -> np.ndarray:
    """Start of each of ``num_parts`` equal contiguous output partitions and
    the end n: partition p holds floor(n/P) elements, plus one when
    p < n mod P (Sec. 1.1; footnote 7 of Sec. 3.4.2).  Returns uint64[P+1]."""
    if num_parts < 1:
        raise ValueError("num_parts must be >= 1")
    q, r = divmod(int(n), int(num_parts))
    p = np.arange(num_parts + 1, dtype=np.uint64)
    return p * np.uint64(q) + np.minimum(p, np.uint64(r))


def sort_segmented(keys, vals, seg_offsets, num_parts: int = 64, kind: str = "u32"):
    """Each segment [seg_offsets[s], seg_offsets[s+1]) sorted on its own
    (stable by key when ``vals`` is given), with the segment's partition
    offsets made absolute by adding the segment start.  Returns
    (keys_out, vals_out or None, part_offsets uint64[num_segs, P+1])."""
    keys = _u32(keys)
    seg_offsets = np.asarray(seg_offsets, dtype=np.uint64)
    nseg = seg_offsets.size - 1
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(_u32(vals))
    po = np.zeros((max(nseg, 0), num_parts + 1), dtype=np.uint64)
    for s in range(nseg):
        a, b = int(seg_offsets[s]), int(seg_offsets[s + 1])
        if vals is None:
            ko[a:b] = sort_keys(keys[a:b], kind)
        else:
            ko[a:b], vo[a:b] = sort_pairs(keys[a:b], _u32(vals)[a:b], kind)
        po[s] = partition_offsets(b - a, num_parts) + np.uint64(a)
    return ko, vo, po


def digit_plan(digit_bits: int, key_bits: int = 32) -> list[tuple[int, int]]:
    """(shift, width) of each digit, least significant first; the last digit
    takes what is left of the key (the paper's global radix splits 31 bits as
    16 + 15, Sec. 5)."""
    out, shift = [], 0
    while shift < key_bits:
        w = min(digit_bits, key_bits - shift)
        out.append((shift, w))
        shift += w
    return out


def digit_of(keys, shift: int, width: int) -> np.ndarray:
    """The bucket index of each key: ``width`` bits starting at ``shift``
    (Sec. 3.2 takes the top log2(buckets) bits with bit operations)."""
    keys = _u32(keys).astype(np.uint64)
    return ((keys >> np.uint64(shift)) & np.uint64((1 << width) - 1)).astype(np.int64)


def digit_histograms(keys, plan: list[tuple[int, int]]) -> list[np.ndarray]:
    """For every digit of ``plan``, how many keys fall in each of its 2^width
    buckets (the count loop of Sec. 3.2).  Returns uint64 arrays."""
    return [np.bincount(digit_of(keys, s, w), minlength=1 << w).astype(np.uint64)
            for s, w in plan]


def digit_bases(hist) -> np.ndarray:
    """Exclusive cumulative totals: base[v] = number of keys whose digit is
    below v, i.e. where bucket v starts in the distributed output (Sec. 3.2,
    Sec. 4.4)."""
    hist = np.asarray(hist, dtype=np.uint64)
    base = np.zeros_like(hist)
    if hist.size > 1:
        base[1:] = np.cumsum(hist[:-1], dtype=np.uint64)
    return base


def skippable_digits(hists, n: int) -> list[bool]:
    """A digit is skippable when one bucket holds all n keys: distributing by
    it leaves every key where it is."""
    return [bool(n > 0 and int(h.max()) == n) or n == 0 for h in hists]


def distribute(keys, vals, shift: int, width: int):
    """One stable distribution pass by a digit: keys grouped by bucket, buckets
    in ascending order, input order kept inside a bucket (Sec. 3.2 partial
    sort; Sec. 3.3.1).  ``vals`` may be None."""
    keys = _u32(keys)
    perm = np.argsort(digit_of(keys, shift, width), kind="stable")
    return keys[perm], (None if vals is None else _u32(vals)[perm])


def lsd_sort(keys, vals, digit_bits: int):
    """The LSD radix sort of Sec. 3.3.1 spelled out: ``distribute`` by each
    digit, least significant first.  Used only to pin ``distribute``; the
    final result is checked against ``sort_keys``/``sort_pairs``."""
    k, v = _u32(keys), (None if vals is None else _u32(vals))
    for s, w in digit_plan(digit_bits):
        k, v = distribute(k, v, s, w)
    return k, v


def msd_buckets(keys, vals, shift: int, width: int):
    """The bucketing phase of Sec. 3.2 on the top digit: the stable
    distribution by that digit plus where each bucket starts and ends.
    Returns (keys, vals, bucket_offsets uint64[2^width + 1])."""
    k, v = distribute(keys, vals, shift, width)
    h = digit_histograms(keys, [(shift, width)])[0]
    offs = np.zeros(h.size + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(h, dtype=np.uint64)
    return k, v, offs


def ordered_words(keys, kind: str = "u32") -> np.ndarray:
    """32-bit words whose unsigned order is the order of ``kind``: unsigned
    words as they are; two's-complement words with the sign bit flipped
    (negative values below non-negative ones); binary32 words in totalOrder
    (IEEE 754-2008 Sec. 5.10): every bit of a word with the sign bit set
    flipped (larger magnitudes first), only the sign bit of the others."""
    w = _u32(keys)
    if kind == "u32":
        return w.copy()
    if kind == "i32":
        return w ^ np.uint32(0x80000000)
    if kind == "f32":
        neg = (w >> np.uint32(31)).astype(bool)
        return np.where(neg, ~w, w | np.uint32(0x80000000)).astype(np.uint32)
    raise ValueError(f"ordered_words covers the 32-bit kinds, not {kind!r}")


def selection_sample(n: int, sample: int = 1000) -> np.ndarray:
    """Positions of the evenly spaced sample (Sec. 4.2.1; footnote 8: 1000
    points): floor(i * n / s) for i < s = min(sample, n)."""
    s = min(sample, n)
    return (np.arange(s, dtype=np.uint64) * np.uint64(n)) // np.uint64(max(s, 1))


def choose_plan(keys, kind: str = "u32", bits: int = 13, sample: int = 1000, cells: int = 64,
                max_problem: int = 2):
    """The selection of Sec. 4.2.1 before a bucketing (MSD) plan.

    Take the evenly spaced sample; bucket each sampled key (in the order of
    ``kind``) by the top ``bits`` of the sample's significant bits; the
    sorted buckets stand for the bucketed output, split into ``cells``
    equal ranges of sample ranks (the output partitions).  Each cell counts
    its sampled elements whose bucket is not above the maximum of its left
    neighbour: those are not separated by the bucketing.  A cell with 65 %
    or more such elements is a problem cell; more than ``max_problem`` of
    them mean the data is clustered and the bucketing plan is abandoned.

    Returns (sorted sample buckets, problem cells, clustered)."""
    w = ordered_words(keys, kind)
    n = w.size
    if n == 0:
        return np.zeros(0, dtype=np.uint32), 0, False
    s = w[selection_sample(n, sample)]
    width = int(s.max()).bit_length()
    shift = max(0, width - bits)
    b = np.sort(s >> np.uint32(shift))
    S = b.size
    problem = 0
    for p in range(1, cells):
        lo, hi = p * S // cells, (p + 1) * S // cells
        if hi <= lo or lo == 0:  # an empty cell, or one with no sampled element to its left
            continue
        left_max = b[lo - 1]
        over = int(np.count_nonzero(b[lo:hi] <= left_max))
        if 100 * over >= 65 * (hi - lo):
            problem += 1
    return b, problem, problem > max_problem
