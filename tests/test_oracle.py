"""Pins of the oracle against things other than itself.

The oracle (``oracle/``) is the definition of the sort written with numpy.
These tests tie it to independent facts:

* brute force: a hand-written stable insertion sort (pure Python) on small
  inputs, and every input of length <= 6 over {0, 1, 2, 2^32-1};
* invariants that together characterise a stable sort: ascending unsigned
  order, the same multiset of keys (per-value counts), payloads of equal keys
  increasing when the payload is the input position;
* the partition rule of Sec. 1.1 / footnote 7 of Sec. 3.4.2: sizes sum to n,
  differ by at most one, and never increase with the partition index, which
  fixes the offsets uniquely; plus hand-worked fixtures under tests/golden/;
* the radix steps of Sec. 3.2 / 3.3.1 against a hand-worked example and
  against brute-force counting and bucket lists, and the LSD theorem (all
  digits distributed low to high give the sorted order);
* planted mistakes: mutated copies of oracle functions must fail the pins.
"""
from __future__ import annotations

import itertools
import os
from collections import Counter

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U32MAX = (1 << 32) - 1


# ---------------------------------------------------------------- brute force
def insertion_sort_pairs(keys, vals):
    """Stable insertion sort on Python ints: an element moves left only past
    strictly greater keys."""
    a = [(int(k), int(v)) for k, v in zip(keys, vals)]
    for i in range(1, len(a)):
        x = a[i]
        j = i - 1
        while j >= 0 and a[j][0] > x[0]:
            a[j + 1] = a[j]
            j -= 1
        a[j + 1] = x
    return [k for k, _ in a], [v for _, v in a]


def brute_histogram(keys, shift, width):
    """The count loop of Sec. 3.2, one element at a time."""
    counts = [0] * (1 << width)
    for k in keys:
        counts[(int(k) >> shift) & ((1 << width) - 1)] += 1
    return counts


def brute_distribute(keys, vals, shift, width):
    """Bucket lists: append each element to its bucket in input order, then
    concatenate the buckets in ascending order."""
    buckets = [[] for _ in range(1 << width)]
    for k, v in zip(keys, vals):
        buckets[(int(k) >> shift) & ((1 << width) - 1)].append((int(k), int(v)))
    flat = [e for b in buckets for e in b]
    return [k for k, _ in flat], [v for _, v in flat]


# ------------------------------------------------------------------- checkers
def check_sort_pairs(fn, keys):
    """Raise AssertionError unless fn(keys, positions) is the stable sort."""
    keys = np.asarray(keys, dtype=np.uint32)
    vals = np.arange(keys.size, dtype=np.uint32)
    ko, vo = fn(keys, vals)
    ko = [int(x) for x in ko]
    vo = [int(x) for x in vo]
    assert len(ko) == keys.size and len(vo) == keys.size
    # ascending unsigned order
    assert all(ko[i] <= ko[i + 1] for i in range(len(ko) - 1))
    # same multiset of keys
    assert Counter(ko) == Counter(int(x) for x in keys)
    # every payload names the key it came with
    assert all(int(keys[v]) == k for k, v in zip(ko, vo))
    # stability: equal keys keep increasing input positions
    assert all(vo[i] < vo[i + 1] for i in range(len(ko) - 1) if ko[i] == ko[i + 1])
    bk, bv = insertion_sort_pairs(keys, vals)
    assert ko == bk and vo == bv


def check_offsets(fn, n, P):
    off = [int(x) for x in fn(n, P)]
    assert len(off) == P + 1 and off[0] == 0 and off[-1] == n
    sizes = [off[i + 1] - off[i] for i in range(P)]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
    assert all(sizes[i] >= sizes[i + 1] for i in range(P - 1))


def read_golden_offsets():
    rows = []
    with open(os.path.join(GOLDEN, "partition_offsets.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            head, tail = line.split("|")
            n, P = (int(x) for x in head.split())
            rows.append((n, P, [int(x) for x in tail.split()]))
    return rows


def read_golden_sorts():
    rows = []
    with open(os.path.join(GOLDEN, "sort_examples.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            fields = [[int(x) for x in part.split()] for part in line.split(";")]
            rows.append(fields)
    return rows


def read_golden_radix():
    d = {}
    with open(os.path.join(GOLDEN, "radix_example.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            d[name] = [int(x) for x in vals]
    return d


# ---------------------------------------------------------------------- tests
def test_golden_sorts():
    for keys, vals, sk, sv in read_golden_sorts():
        ko, vo = oracle.sort_pairs(np.array(keys, np.uint32), np.array(vals, np.uint32))
        assert list(ko) == sk and list(vo) == sv
        assert list(oracle.sort_keys(np.array(keys, np.uint32))) == sk


def test_golden_offsets():
    rows = read_golden_offsets()
    assert len(rows) >= 10
    for n, P, want in rows:
        assert [int(x) for x in oracle.partition_offsets(n, P)] == want, (n, P)


def test_golden_radix_steps():
    g = read_golden_radix()
    keys = np.array(g["keys"], np.uint32)
    vals = np.array(g["vals"], np.uint32)
    h0, h1 = oracle.digit_histograms(keys, [(0, 2), (2, 2)])
    assert list(h0) == g["hist0"] and list(h1) == g["hist1"]
    assert list(oracle.digit_bases(h0)) == g["base0"]
    assert list(oracle.digit_bases(h1)) == g["base1"]
    k0, v0 = oracle.distribute(keys, vals, 0, 2)
    assert list(k0) == g["pass0_keys"] and list(v0) == g["pass0_vals"]
    k1, v1 = oracle.distribute(k0, v0, 2, 2)
    assert list(k1) == g["pass1_keys"] and list(v1) == g["pass1_vals"]


def test_exhaustive_tiny():
    alphabet = [0, 1, 2, U32MAX]
    count = 0
    for n in range(0, 7):
        for tup in itertools.product(alphabet, repeat=n):
            check_sort_pairs(oracle.sort_pairs, tup)
            count += 1
    assert count == sum(4 ** n for n in range(7))


@pytest.mark.parametrize("dist", ["uniform", "few", "equal", "sorted", "reverse", "two", "topbit"])
def test_bruteforce_small(dist):
    rng_keys = synth.uniform31(2048, 1234).astype(np.uint64)
    n = 2048 if dist != "uniform" else 1500
    if dist == "uniform":
        keys = rng_keys[:n] | (rng_keys[:n] << np.uint64(1)) & np.uint64(U32MAX)
    elif dist == "few":
        keys = rng_keys % np.uint64(7)
    elif dist == "equal":
        keys = np.full(n, 123456789, np.uint64)
    elif dist == "sorted":
        keys = np.sort(rng_keys)
    elif dist == "reverse":
        keys = np.sort(rng_keys)[::-1]
    elif dist == "two":
        keys = np.where(rng_keys & np.uint64(1), np.uint64(U32MAX), np.uint64(0))
    else:  # values straddling 2^31: catches a signed comparison
        keys = (np.uint64(1 << 31) - np.uint64(1024)) + rng_keys % np.uint64(2048)
    check_sort_pairs(oracle.sort_pairs, keys.astype(np.uint32))
    ko = oracle.sort_keys(keys.astype(np.uint32))
    bk, _ = insertion_sort_pairs(keys, range(keys.size))
    assert [int(x) for x in ko] == bk


@pytest.mark.parametrize("name", sorted(synth.DISTRIBUTIONS))
def test_invariants_each_distribution(name):
    keys = synth.DISTRIBUTIONS[name](1 << 15, 99)
    vals = np.arange(keys.size, dtype=np.uint32)
    ko, vo = oracle.sort_pairs(keys, vals)
    assert np.all(ko[:-1] <= ko[1:])
    assert np.array_equal(keys[vo], ko)
    assert np.array_equal(np.sort(vo), vals)  # vals is a permutation
    eq = ko[:-1] == ko[1:]
    assert np.all(vo[:-1][eq] < vo[1:][eq])
    assert Counter(ko.tolist()) == Counter(keys.tolist())


@pytest.mark.parametrize("P", [1, 2, 3, 7, 63, 64, 65, 1000])
def test_offsets_invariants(P):
    for n in list(range(0, 3 * P + 3)) + [1 << 20, (1 << 26) + 7, (1 << 32) - 1]:
        check_offsets(oracle.partition_offsets, n, P)


def test_histograms_and_bases_bruteforce():
    keys = synth.uniform31(4000, 7).astype(np.uint32) | np.uint32(1 << 31)
    for plan in (oracle.digit_plan(8), oracle.digit_plan(11), [(5, 3), (0, 1)]):
        hs = oracle.digit_histograms(keys, plan)
        for (s, w), h in zip(plan, hs):
            assert [int(x) for x in h] == brute_histogram(keys, s, w)
            assert int(h.sum()) == keys.size
            b = oracle.digit_bases(h)
            dig = [(int(k) >> s) & ((1 << w) - 1) for k in keys]
            cnt = Counter(dig)
            # base[v] = number of keys whose digit is below v
            running = 0
            for v in range(1 << w):
                assert int(b[v]) == running
                running += cnt.get(v, 0)


def test_digit_plan():
    assert oracle.digit_plan(8) == [(0, 8), (8, 8), (16, 8), (24, 8)]
    assert oracle.digit_plan(11) == [(0, 11), (11, 11), (22, 10)]
    assert oracle.digit_plan(16, 31) == [(0, 16), (16, 15)]  # the 16+15 of Sec. 5


def test_distribute_bruteforce_and_lsd_theorem():
    keys = synth.gauss_mix(3000, 5)
    vals = np.arange(keys.size, dtype=np.uint32)
    for s, w in [(0, 8), (8, 8), (22, 10), (0, 11), (3, 5)]:
        k, v = oracle.distribute(keys, vals, s, w)
        bk, bv = brute_distribute(keys, vals, s, w)
        assert [int(x) for x in k] == bk and [int(x) for x in v] == bv
    sk, sv = oracle.sort_pairs(keys, vals)
    for bits in (1, 4, 8, 11, 13, 16):
        k, v = oracle.lsd_sort(keys, vals, bits)
        assert np.array_equal(k, sk) and np.array_equal(v, sv), bits


def check_msd_offsets(keys, k, offs, shift, width):
    """Bucket b of the bucketing phase (Sec. 3.2) holds exactly the keys whose
    top digit is b: its size is the brute-force count of that digit, and every
    key inside its range carries that digit."""
    counts = brute_histogram(keys, shift, width)
    assert offs.size == (1 << width) + 1 and int(offs[0]) == 0
    for b in range(1 << width):
        a, e = int(offs[b]), int(offs[b + 1])
        assert e - a == counts[b], b
        assert all(((int(x) >> shift) & ((1 << width) - 1)) == b for x in k[a:e]), b


@pytest.mark.parametrize("dist,n,shift,width", [
    ("tight_clusters", 5000, 21, 11), ("uniform31", 3000, 18, 13), ("few_distinct", 2000, 20, 12),
])
def test_msd_buckets_then_local_sort(dist, n, shift, width):
    keys = getattr(synth, dist)(n, 3)
    vals = np.arange(keys.size, dtype=np.uint32)
    k, v, offs = oracle.msd_buckets(keys, vals, shift, width)
    assert int(offs[0]) == 0 and int(offs[-1]) == keys.size
    check_msd_offsets(keys, k, offs, shift, width)
    # sorting each bucket on its own gives the full stable sort
    outk, outv = k.copy(), v.copy()
    for b in range(offs.size - 1):
        a, e = int(offs[b]), int(offs[b + 1])
        outk[a:e], outv[a:e] = oracle.sort_pairs(k[a:e], v[a:e])
    sk, sv = oracle.sort_pairs(keys, vals)
    assert np.array_equal(outk, sk) and np.array_equal(outv, sv)


def test_msd_offsets_pin_catches_shifted_bases():
    """A plausible mistake: the bucket offsets taken as the exclusive bases
    shifted by one slot.  On clustered keys the top bucket is empty, so the
    last offset still equals n; the per-bucket check must still fail."""
    keys = synth.tight_clusters(5000, 3)
    vals = np.arange(keys.size, dtype=np.uint32)
    k, _, offs = oracle.msd_buckets(keys, vals, 21, 11)
    wrong = np.zeros_like(offs)
    wrong[1:] = oracle.digit_bases(oracle.digit_histograms(keys, [(21, 11)])[0])
    assert int(wrong[0]) == 0 and int(wrong[-1]) == keys.size  # the ends alone do not see it
    with pytest.raises(AssertionError):
        check_msd_offsets(keys, k, wrong, 21, 11)


def test_skippable_digits():
    keys = (synth.uniform31(1000, 1) & np.uint32(0x3FF)) | np.uint32(0x5 << 24)
    plan = oracle.digit_plan(8)
    sk = oracle.skippable_digits(oracle.digit_histograms(keys, plan), keys.size)
    assert sk == [False, False, True, True]
    for (s, w), skip in zip(plan, sk):
        if skip:  # distributing by a skippable digit moves nothing
            k, _ = oracle.distribute(keys, None, s, w)
            assert np.array_equal(k, keys)


def test_segmented_bruteforce():
    sizes = [0, 1, 5, 0, 40, 3, 0]
    offs = np.zeros(len(sizes) + 1, np.uint64)
    offs[1:] = np.cumsum(sizes)
    n = int(offs[-1])
    keys = (synth.uniform31(n, 17) % np.uint32(9)).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    ko, vo, po = oracle.sort_segmented(keys, vals, offs, num_parts=4)
    for s in range(len(sizes)):
        a, b = int(offs[s]), int(offs[s + 1])
        bk, bv = insertion_sort_pairs(keys[a:b], vals[a:b])
        assert [int(x) for x in ko[a:b]] == bk and [int(x) for x in vo[a:b]] == bv
        assert int(po[s, 0]) == a and int(po[s, -1]) == b
        check_offsets(lambda m, P: po[s] - np.uint64(a), b - a, 4)
    ko2, vo2, _ = oracle.sort_segmented(keys, None, offs, num_parts=4)
    assert vo2 is None and np.array_equal(ko2, ko)


# ------------------------------------------------------------ planted mistakes
def _mut_signed(keys, vals):
    perm = np.argsort(keys.astype(np.int32), kind="stable")
    return keys[perm], vals[perm]


def _mut_unstable(keys, vals):
    # reverse the input, then stable sort: equal keys come out reversed
    r = keys[::-1]
    perm = np.argsort(r, kind="stable")
    return r[perm], vals[::-1][perm]


def _mut_drop(keys, vals):
    k, v = oracle.sort_pairs(keys, vals)
    if k.size:
        k, v = k.copy(), v.copy()
        k[-1], v[-1] = k[0], v[0]
    return k, v


def _mut_offsets_upper(n, P):
    q, r = divmod(n, P)
    sizes = [q + (1 if p >= P - r else 0) for p in range(P)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)


def _mut_bases_inclusive(h):
    return np.cumsum(np.asarray(h, np.uint64))


@pytest.mark.parametrize("mut", [_mut_signed, _mut_unstable, _mut_drop])
def test_planted_sort_mistakes_are_caught(mut):
    caught = False
    for keys in ([U32MAX, 0, 1 << 31, 5], [2, 1, 2, 1, 2], [3, 1, 2, 1]):
        try:
            check_sort_pairs(mut, keys)
        except AssertionError:
            caught = True
    assert caught


def test_planted_offset_and_base_mistakes_are_caught():
    with pytest.raises(AssertionError):
        check_offsets(_mut_offsets_upper, 10, 4)
    h = oracle.digit_histograms(np.array([13, 6, 9, 2, 14, 5], np.uint32), [(0, 2)])[0]
    assert list(_mut_bases_inclusive(h)) != read_golden_radix()["base0"]


# ------------------------------------------------------------ key kinds
def read_golden_key_kinds():
    rows = []
    with open(os.path.join(GOLDEN, "key_kinds.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kind, a, b = (part.strip() for part in line.split(";"))
            dt = np.uint64 if kind.endswith("64") else np.uint32
            rows.append((kind, np.array([int(x, 16) for x in a.split()], dt),
                         np.array([int(x, 16) for x in b.split()], dt)))
    return rows


def test_golden_key_kinds():
    for kind, words, want in read_golden_key_kinds():
        assert np.array_equal(oracle.sort_keys(words, kind), want), kind


def _random_words(n, seed):
    return synth.splitmix64(seed, n).astype(np.uint64).view(np.uint32)[::2].copy()


def test_i32_order_is_python_integer_order():
    w = np.concatenate([_random_words(3000, 5), np.array([0, 1, 0xFFFFFFFF, 0x80000000, 0x7FFFFFFF], np.uint32)])
    w = np.concatenate([w, w[:500]])  # duplicates
    ints = [int(x) - (1 << 32) if x >= 1 << 31 else int(x) for x in w]
    want = sorted(range(len(ints)), key=lambda i: ints[i])  # Python's sort is stable
    assert np.array_equal(oracle.order_perm(w, "i32"), np.array(want))


def _floats_without_nan_or_signed_zero(n, seed):
    w = _random_words(n, seed)
    keep = ((w & np.uint32(0x7F800000)) != np.uint32(0x7F800000)) | ((w & np.uint32(0x007FFFFF)) == 0)  # no NaN
    keep &= (w & np.uint32(0x7FFFFFFF)) != 0  # no zero of either sign
    w = w[keep]
    return np.concatenate([w, w[: w.size // 4], np.array([0x7F800000, 0xFF800000], np.uint32)])


def test_f32_order_is_numeric_order_off_nan_and_zero():
    """Away from NaNs and zeros, totalOrder is the numeric order of the
    values (numpy's float comparison), ties kept in input order."""
    w = _floats_without_nan_or_signed_zero(5000, 6)
    want = np.argsort(w.view(np.float32), kind="stable")
    assert np.array_equal(oracle.order_perm(w, "f32"), want)


def test_f32_order_sign_nan_and_zero_rules():
    w = _random_words(20000, 7)  # about 0.4 % NaNs of each sign
    w = np.concatenate([w, np.array([0x00000000, 0x80000000, 0x7F800000, 0xFF800000], np.uint32)])
    s = oracle.sort_keys(w, "f32")
    neg = (s >> np.uint32(31)).astype(bool)
    assert not np.any(~neg[:-1] & neg[1:]), "a word with the sign bit set after one without"
    f = s.view(np.float32)
    nan = np.isnan(f)
    # negative NaNs first, positive NaNs last, -0 right before +0
    first_num = int(np.argmax(~nan))
    assert np.all(nan[:first_num]) and np.all(neg[:first_num])
    last_num = len(s) - int(np.argmax(~nan[::-1]))
    assert np.all(nan[last_num:]) and not np.any(neg[last_num:])
    iz = int(np.flatnonzero(s == np.uint32(0x80000000))[0])
    assert s[iz + 1] == 0 and not np.any(f[:iz][~nan[:iz]] > 0)


def _mut_f32_magnitudes_not_reversed(w):
    negative = (w >> np.uint32(31)).astype(bool)
    magnitude = (w & np.uint32(0x7FFFFFFF)).astype(np.int64)
    return np.lexsort((magnitude, np.where(negative, 0, 1)))


def _mut_f32_as_unsigned(w):
    return np.argsort(w, kind="stable")


@pytest.mark.parametrize("mut", [_mut_f32_magnitudes_not_reversed, _mut_f32_as_unsigned])
def test_planted_f32_mistakes_are_caught(mut):
    w = _floats_without_nan_or_signed_zero(5000, 6)
    assert not np.array_equal(mut(w), np.argsort(w.view(np.float32), kind="stable"))
    golden = [(k, a, b) for k, a, b in read_golden_key_kinds() if k == "f32"]
    assert any(not np.array_equal(a[mut(a)], b) for _, a, b in golden)


def test_i64_order_is_python_integer_order():
    w = synth.splitmix64(8, 3000)
    w = np.concatenate([w, w[:400], np.array([0, 1, 2**64 - 1, 2**63, 2**63 - 1], np.uint64)])
    ints = [int(x) - (1 << 64) if x >= 1 << 63 else int(x) for x in w]
    want = sorted(range(len(ints)), key=lambda i: ints[i])
    assert np.array_equal(oracle.order_perm(w, "i64"), np.array(want))
    assert np.array_equal(oracle.order_perm(w, "u64"), np.array(sorted(range(len(w)), key=lambda i: int(w[i]))))


def test_f64_order_is_numeric_order_off_nan_and_zero():
    w = synth.splitmix64(9, 6000)
    exp = (w >> np.uint64(52)) & np.uint64(0x7FF)
    keep = (exp != 0x7FF) & ((w & np.uint64(2**63 - 1)) != 0)
    w = w[keep]
    w = np.concatenate([w, w[: w.size // 4], np.array([0x7FF0000000000000, 0xFFF0000000000000], np.uint64)])
    assert np.array_equal(oracle.order_perm(w, "f64"), np.argsort(w.view(np.float64), kind="stable"))


# ------------------------------------------------------------ merge
def _two_pointer_merge(a, b, va, vb, before):
    """The textbook merge of two sorted lists, taking from a while its head
    does not come after b's head (``before(x, y)``: x strictly precedes y)."""
    i = j = 0
    keys, vals = [], []
    while i < len(a) or j < len(b):
        if j >= len(b) or (i < len(a) and not before(b[j], a[i])):
            keys.append(a[i]); vals.append(va[i]); i += 1
        else:
            keys.append(b[j]); vals.append(vb[j]); j += 1
    return keys, vals


@pytest.mark.parametrize("kind", ["u32", "i32"])
@pytest.mark.parametrize("sizes", [(0, 0), (0, 3), (4, 0), (1, 1), (50, 7), (200, 300)])
def test_merge_is_the_textbook_merge(kind, sizes):
    na, nb = sizes
    a = oracle.sort_keys(synth.uniform31(na, 1) % np.uint32(20), kind) if na else np.zeros(0, np.uint32)
    b = oracle.sort_keys(synth.uniform31(nb, 2) % np.uint32(20), kind) if nb else np.zeros(0, np.uint32)
    if kind == "i32":  # negative keys too
        a = oracle.sort_keys((a.view(np.int32) - 10).view(np.uint32), kind)
        b = oracle.sort_keys((b.view(np.int32) - 10).view(np.uint32), kind)
    va = np.arange(na, dtype=np.uint32)
    vb = np.arange(na, na + nb, dtype=np.uint32)
    conv = (lambda w: int(np.uint32(w).view(np.int32))) if kind == "i32" else int
    wk, wv = _two_pointer_merge([conv(x) for x in a], [conv(x) for x in b], list(va), list(vb),
                                lambda x, y: x < y)
    ko, vo = oracle.merge(a, b, va, vb, kind)
    assert [conv(x) for x in ko] == wk and list(vo) == wv


# ---------------------------------------------- the selection of Sec. 4.2.1
def read_golden_selection():
    cases, cur = [], None
    for line in open(os.path.join(GOLDEN, "selection_example.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line == "case":
            cur = {}
            cases.append(cur)
            continue
        k, *v = line.split()
        cur[k] = [int(x) for x in v]
    return cases


def test_golden_selection_examples():
    cases = read_golden_selection()
    assert len(cases) == 4
    for c in cases:
        b, problem, clustered = oracle.choose_plan(np.array(c["keys"], dtype=np.uint32), "u32", bits=c["bits"][0],
                                                   sample=c["sample"][0], cells=c["cells"][0],
                                                   max_problem=c["max_problem"][0])
        assert [int(x) for x in b] == c["buckets"], c
        assert problem == c["problem"][0] and int(clustered) == c["clustered"][0], c


def test_selection_sample_positions_are_evenly_spaced():
    assert list(oracle.selection_sample(12, 4)) == [0, 3, 6, 9]
    assert list(oracle.selection_sample(5, 1000)) == [0, 1, 2, 3, 4]  # fewer keys than the sample: all of them
    pos = oracle.selection_sample(10 ** 9, 1000)
    assert pos.size == 1000 and pos[0] == 0 and np.all(np.diff(pos.astype(np.int64)) >= 10 ** 6 - 1)


def test_ordered_words_give_each_kinds_order():
    rng = np.random.default_rng(3)
    w = rng.integers(0, 1 << 32, 5000, dtype=np.uint64).astype(np.uint32)
    w[:8] = [0, 1, 0x7FFFFFFF, 0x80000000, 0x80000001, 0xFFFFFFFF, 0x7F800000, 0xFF800000]
    for kind in ("u32", "i32", "f32"):
        o = oracle.ordered_words(w, kind)
        assert np.array_equal(np.argsort(o, kind="stable"), oracle.order_perm(w, kind)), kind


def test_selection_threshold_is_65_percent_inclusive():
    """A cell of 20 sampled elements with 13 in its left neighbour's last
    bucket (65 %) is a problem cell; with 12 (60 %) it is not."""
    for copies, want in ((14, 1), (13, 0)):
        keys = np.concatenate([np.arange(19), np.full(copies, 19), np.arange(100, 100 + 40 - 19 - copies)])
        keys = keys.astype(np.uint32)
        assert keys.size == 40
        _, problem, _ = oracle.choose_plan(keys, bits=32, sample=40, cells=2, max_problem=0)
        assert problem == want, copies


def test_selection_on_the_workloads():
    """Uniform keys spread over the buckets: no problem cell.  Tight clusters
    (eight windows of 4096 values) cannot be separated by 13-bit buckets:
    most cells are problem cells and the bucketing plan is abandoned, as for
    the paper's fifth data set.  Equal keys: every cell after the first."""
    n = 1 << 18
    _, p, c = oracle.choose_plan(synth.uniform31(n, 1))
    assert p == 0 and not c
    _, p, c = oracle.choose_plan(synth.tight_clusters(n, 1))
    assert p > 2 and c
    _, p, c = oracle.choose_plan(np.full(5000, 77, np.uint32))
    assert p == 63 and c
    # all sampled keys distinct and buckets as fine as the keys: no overlap
    _, p, _ = oracle.choose_plan(np.arange(5000, dtype=np.uint32) * np.uint32(7), bits=32)
    assert p == 0


def test_selection_with_fewer_sampled_keys_than_cells():
    """With fewer sampled keys than cells, most cells are empty and the first
    non-empty one starts at rank 0: it has no left neighbour to overlap."""
    _, p, _ = oracle.choose_plan(np.array([5], np.uint32))
    assert p == 0
    _, p, _ = oracle.choose_plan(np.array([5, 5], np.uint32))  # cells 31 (rank 0) and 63 (rank 1)
    assert p == 1


@pytest.mark.parametrize("threads", [1, 3, 16])
def test_cpu_radix_baseline_matches_the_oracle(threads):
    """The all-core CPU baseline (C, not the oracle) sorts like the oracle:
    empty, tiny, ragged chunk counts, equal keys, extreme words."""
    from oracle import cpu_baseline
    rng = np.random.default_rng(threads)
    cases = [np.zeros(0, np.uint32), np.array([7], np.uint32), synth.uniform31(5, 2),
             rng.integers(0, 1 << 32, 100_003, dtype=np.uint64).astype(np.uint32),
             synth.few_distinct(70_001, 3), np.full(50_000, 0xFFFFFFFF, np.uint32),
             np.array([0xFFFFFFFF, 0, 0x80000000, 0x7FFFFFFF, 1] * 9000, np.uint32)]
    for keys in cases:
        assert np.array_equal(cpu_baseline.sort(keys, threads), oracle.sort_keys(keys))
