"""The seeded workloads have the properties the paper's data-set table
(Sec. 1.1) asks of their stand-ins, and are reproducible."""
import numpy as np

import synth


def test_splitmix64_known_values():
    # SplitMix64 with seed 0: the first outputs of the published generator
    z = synth.splitmix64(0, 3)
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform31_range_and_determinism():
    a = synth.uniform31(1 << 16, 5)
    assert a.dtype == np.uint32 and int(a.max()) < (1 << 31)
    assert np.array_equal(a, synth.uniform31(1 << 16, 5))
    assert not np.array_equal(a, synth.uniform31(1 << 16, 6))
    # roughly uniform: each top-4-bit bucket within 5% of n/16
    h = np.bincount(a >> 27, minlength=16)
    assert np.all(np.abs(h - a.size / 16) < 0.05 * a.size / 16)


def test_skewed_chunks():
    n = 1 << 20
    s = synth.skewed_chunk_sizes(n, 64, 3)
    assert s.size == 64 and int(s.sum()) == n
    assert int(s.max()) == n // 8 and np.sum(s == s.max()) == 1
    k = synth.skewed_chunks(n, 3)
    assert k.size == n and int(k.max()) < (1 << 31)


def test_few_distinct():
    k = synth.few_distinct(1 << 20, 4)
    assert np.unique(k).size <= 65536 and np.unique(k).size > 65000


def test_gauss_mix_and_tight_clusters():
    k = synth.gauss_mix(1 << 18, 8)
    assert int(k.max()) < (1 << 31)
    t = synth.tight_clusters(1 << 18, 8)
    u = np.unique(t)
    assert u.size <= 8 * 4096
    # split the distinct values at gaps of 4096 or more: at most 8 groups
    groups = 1 + int(np.sum(np.diff(u.astype(np.int64)) >= 4096))
    assert groups <= 8


def test_segment_sizes():
    s = synth.segment_sizes(9)
    assert s.size <= 4096 and int(s.sum()) <= (1 << 28)
    assert int(s.min()) >= 1024 and int(s.max()) <= (1 << 20)
    k, v, offs = synth.segmented_batch(9, max_segments=50)
    assert int(offs[-1]) == k.size == v.size


def test_serving_requests():
    r = synth.serving_requests(200, 1, rate_per_s=100.0)
    assert len(r) == 200 and r[0]["arrival_s"] == 0.0
    assert all(r[i]["arrival_s"] <= r[i + 1]["arrival_s"] for i in range(199))
    assert all((1 << 16) <= q["n"] <= (1 << 26) for q in r)
    frac = sum(q["pairs"] for q in r) / 200
    assert 0.35 < frac < 0.65
