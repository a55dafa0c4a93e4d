"""Property-based pins of the oracle (hypothesis; skipped where it is not
installed): on arbitrary inputs, the oracle's results satisfy the properties
that define them, checked with plain Python code that shares nothing with
the oracle's numpy formulation."""
import numpy as np
import pytest

import oracle

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

U32 = st.integers(min_value=0, max_value=2**32 - 1)
SETTINGS = dict(max_examples=200, deadline=None)


@settings(**SETTINGS)
@given(st.lists(U32, max_size=300))
def test_sort_pairs_is_the_stable_sort(keys):
    """Sorted by key, payloads of equal keys in input order, a permutation."""
    k = np.array(keys, dtype=np.uint32)
    v = np.arange(len(keys), dtype=np.uint32)
    ko, vo = oracle.sort_pairs(k, v)
    want = sorted(range(len(keys)), key=lambda i: keys[i])  # Python's sort is stable
    assert list(vo) == want
    assert list(ko) == [keys[i] for i in want]


@settings(**SETTINGS)
@given(st.integers(min_value=0, max_value=10**7), st.integers(min_value=1, max_value=300))
def test_partition_offsets_split_evenly_lower_first(n, parts):
    off = [int(x) for x in oracle.partition_offsets(n, parts)]
    sizes = [off[i + 1] - off[i] for i in range(parts)]
    assert off[0] == 0 and off[-1] == n
    assert max(sizes) - min(sizes) <= 1
    assert sizes == sorted(sizes, reverse=True)  # the larger slices come first


@settings(**SETTINGS)
@given(st.lists(U32, max_size=200), st.sampled_from([(0, 8), (8, 8), (24, 8), (0, 11), (21, 11), (3, 5)]))
def test_distribute_groups_by_digit_stably(keys, dig):
    shift, width = dig
    k = np.array(keys, dtype=np.uint32)
    v = np.arange(len(keys), dtype=np.uint32)
    ko, vo = oracle.distribute(k, v, shift, width)
    d = lambda x: (x >> shift) & ((1 << width) - 1)  # noqa: E731
    want = sorted(range(len(keys)), key=lambda i: d(keys[i]))
    assert list(vo) == want and list(ko) == [keys[i] for i in want]


@settings(**SETTINGS)
@given(st.lists(U32, max_size=200), st.sampled_from([8, 11]))
def test_lsd_sort_reaches_the_sort(keys, bits):
    k = np.array(keys, dtype=np.uint32)
    v = np.arange(len(keys), dtype=np.uint32)
    ko, vo = oracle.lsd_sort(k, v, bits)
    want = sorted(range(len(keys)), key=lambda i: keys[i])
    assert list(vo) == want and list(ko) == [keys[i] for i in want]


@settings(**SETTINGS)
@given(st.lists(st.integers(min_value=-2**31, max_value=2**31 - 1), max_size=200))
def test_i32_order(ints):
    w = np.array(ints, dtype=np.int64).astype(np.int32).view(np.uint32)
    assert [int(x) for x in oracle.sort_keys(w, "i32").view(np.int32)] == sorted(ints)


@settings(**SETTINGS)
@given(st.lists(st.floats(width=32, allow_nan=False), max_size=200))
def test_f32_order_is_numeric_with_negative_zero_first(vals):
    w = np.array(vals, dtype=np.float32).view(np.uint32)
    got = oracle.sort_keys(w, "f32")
    f = got.view(np.float32)
    assert np.all(f[1:] >= f[:-1])  # numeric order (-0 == +0 numerically)
    neg = (got >> np.uint32(31)).astype(bool)
    zero = f == 0
    # among the zeros, every -0 comes before every +0
    zs = neg[zero]
    assert np.all(zs[:-1] >= zs[1:])


@settings(**SETTINGS)
@given(st.lists(U32, max_size=150), st.lists(U32, max_size=150))
def test_merge_is_the_stable_sort_of_the_concatenation(a, b):
    a, b = sorted(a), sorted(b)
    va = list(range(len(a)))
    vb = list(range(len(a), len(a) + len(b)))
    ko, vo = oracle.merge(np.array(a, np.uint32), np.array(b, np.uint32), np.array(va, np.uint32),
                          np.array(vb, np.uint32))
    keys, vals = a + b, va + vb
    want = sorted(range(len(keys)), key=lambda i: keys[i])
    assert list(vo) == [vals[i] for i in want] and list(ko) == [keys[i] for i in want]


U64 = st.integers(min_value=0, max_value=2**64 - 1)


@settings(**SETTINGS)
@given(st.lists(st.integers(min_value=-2**63, max_value=2**63 - 1), max_size=200))
def test_i64_order(ints):
    w = np.array(ints, dtype=np.int64).view(np.uint64)
    assert [int(x) for x in oracle.sort_keys(w, "i64").view(np.int64)] == sorted(ints)


@settings(**SETTINGS)
@given(st.lists(st.floats(width=64, allow_nan=False), max_size=200))
def test_f64_order_is_numeric_with_negative_zero_first(vals):
    w = np.array(vals, dtype=np.float64).view(np.uint64)
    got = oracle.sort_keys(w, "f64")
    f = got.view(np.float64)
    assert np.all(f[1:] >= f[:-1])
    neg = (got >> np.uint64(63)).astype(bool)
    zs = neg[f == 0]
    assert np.all(zs[:-1] >= zs[1:])  # every -0 before every +0
    assert sorted(got.tolist()) == sorted(w.tolist())  # a permutation of the words


@settings(**SETTINGS)
@given(st.lists(st.tuples(U64, U64), max_size=200))
def test_u64_pairs_carry_64_bit_values_stably(pairs):
    keys = np.array([k for k, _ in pairs], dtype=np.uint64)
    vals = np.array([v for _, v in pairs], dtype=np.uint64)
    ko, vo = oracle.sort_pairs(keys, vals, "u64")
    want = sorted(range(len(pairs)), key=lambda i: pairs[i][0])  # Python's sort is stable
    assert [int(x) for x in ko] == [pairs[i][0] for i in want]
    assert [int(x) for x in vo] == [pairs[i][1] for i in want]
    assert vo.dtype == np.uint64
