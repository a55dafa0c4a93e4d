"""Parity of the batched segmented sort and of the MSD plan with the oracle
(bit-exact).  Segments of every class are mixed in one call: empty, single
keys, tiny (<= 4096 keys, one 256-thread block), small (<= 16384, one
1024-thread block) and large (tiled passes whose lookback stays inside the
segment).  The MSD plan buckets by the keys' bits 18-31 (2^14 buckets; keys
only: one counting read and one distribution pass; key+value: two stable
passes), then sorts every bucket through the same segmented pipeline (Sec. 3 /
Sec. 4.6: bucketing, then a local radix sort per bucket)."""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu import to_dev, to_host_u32, to_host_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_cs_0004013_gb300 as r
    return r


def _segmented(rs, keys, sizes, pairs, num_parts=64):
    import torch
    offs = np.zeros(len(sizes) + 1, np.uint64)
    offs[1:] = np.cumsum(sizes)
    vals = np.arange(keys.size, dtype=np.uint32)
    ko, vo, po = rs.sort_segmented(to_dev(keys), to_dev(vals) if pairs else None, offs, num_parts=num_parts)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv, wp = oracle.sort_segmented(keys, vals if pairs else None, offs, num_parts)
    assert np.array_equal(to_host_u32(ko), wk)
    if pairs:
        assert np.array_equal(to_host_u32(vo), wv)
    assert np.array_equal(to_host_u64(po).reshape(len(sizes), num_parts + 1), wp)


@pytest.mark.parametrize("pairs", [False, True])
def test_segmented_all_classes(rs, pairs):
    # around the tiled passes' tile sizes too (12,288 keys, 11,264 pairs)
    sizes = [0, 1, 2, 31, 4095, 4096, 4097, 0, 16383, 16384, 16385, 8192 * 3 + 5, 100_000, 1, 7, 250_001, 33,
             3 * 12288 - 1, 3 * 12288 + 1, 2 * 11264 - 1, 2 * 11264, 2 * 11264 + 1]
    n = int(sum(sizes))
    _segmented(rs, synth.gauss_mix(n, 5), sizes, pairs)


@pytest.mark.parametrize("dist", ["uniform", "tight_clusters", "few_distinct"])
def test_segmented_log_uniform_batch(rs, dist):
    sizes = synth.segment_sizes(77, max_segments=300, cap=1 << 24)
    n = int(sizes.sum())
    keys = synth.DISTRIBUTIONS[dist](n, 78)
    _segmented(rs, keys, list(sizes), pairs=True)


def test_segmented_many_small(rs):
    sizes = list((synth.uniform31(5000, 3) % np.uint32(3000)).astype(np.int64))
    n = int(sum(sizes))
    _segmented(rs, synth.uniform31(n, 4) | np.uint32(1 << 31), sizes, pairs=True, num_parts=3)


def test_segmented_one_huge(rs):
    n = (1 << 22) + 77
    _segmented(rs, synth.uniform31(n, 9), [n], pairs=True)


@pytest.mark.parametrize("n", [1, 100, 4096, 65536, 65537, (1 << 20), (1 << 20) + 3, 1 << 22])
@pytest.mark.parametrize("pairs", [False, True])
def test_msd_plan_sizes(rs, n, pairs):
    import torch
    keys = synth.uniform31(n, n) | (synth.uniform31(n, n + 1) << np.uint32(1))
    plan = {"digit_bits": 8, "mode": rs.RS_MODE_MSD}
    if pairs:
        vals = np.arange(n, dtype=np.uint32)
        ko, vo, offs = rs.sort_pairs(to_dev(keys), to_dev(vals), plan=plan)
        torch.cuda.synchronize()
        wk, wv = oracle.sort_pairs(keys, vals)
        assert np.array_equal(to_host_u32(vo), wv)
    else:
        ko, offs = rs.sort(to_dev(keys), plan=plan)
        torch.cuda.synchronize()
        wk = oracle.sort_keys(keys)
    rs.rs_check_device_error()
    assert np.array_equal(to_host_u32(ko), wk)
    assert np.array_equal(offs, oracle.partition_offsets(n, 64))


@pytest.mark.parametrize("dist", sorted(synth.DISTRIBUTIONS))
def test_msd_plan_distributions(rs, dist):
    import torch
    n = 1 << 22
    keys = synth.DISTRIBUTIONS[dist](n, synth.CONFIG_SEED + 3)
    vals = np.arange(n, dtype=np.uint32)
    ko, vo, _ = rs.sort_pairs(to_dev(keys), to_dev(vals), plan={"mode": rs.RS_MODE_MSD})
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv = oracle.sort_pairs(keys, vals)
    assert np.array_equal(to_host_u32(ko), wk)
    assert np.array_equal(to_host_u32(vo), wv)


@pytest.mark.parametrize("dist", sorted(synth.DISTRIBUTIONS))
def test_msd_plan_full_size_distributions(rs, dist):
    """The MSD plan at the workload size, 2^26 keys, keys only and with
    payload = input position, for every distribution (tight clusters put
    each cluster in one oversized bucket, sorted by tiled passes)."""
    import torch
    n = 1 << 26
    keys = synth.config_keys(3, dist=dist) if dist != "uniform" else synth.config_keys(2)
    plan = {"digit_bits": 8, "mode": rs.RS_MODE_MSD}
    d = to_dev(keys)
    ko, offs = rs.sort(d, plan=plan)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk = oracle.sort_keys(keys)
    assert np.array_equal(to_host_u32(ko), wk)
    assert np.array_equal(offs, oracle.partition_offsets(n, 64))
    del ko
    vals = np.arange(n, dtype=np.uint32)
    ko, vo, _ = rs.sort_pairs(d, to_dev(vals), plan=plan)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk2, wv = oracle.sort_pairs(keys, vals)
    assert np.array_equal(to_host_u32(ko), wk2)
    assert np.array_equal(to_host_u32(vo), wv)


def test_msd_bucket_boundaries(rs):
    """Keys on both sides of every bucket boundary (bit 18), the lowest and
    the highest bucket, and signed keys (the bucket is taken on the order map)."""
    import torch
    b = np.arange(0, 1 << 14, 37, dtype=np.uint64) << np.uint64(18)
    bi = b.astype(np.int64)
    keys = np.concatenate([bi, bi - 1, bi + 1, [0, 1, 0xFFFFFFFF, 0xFFFC0000]]) & 0xFFFFFFFF
    keys = np.tile(keys.astype(np.uint32), 9)
    for kind, code in (("u32", 0), ("i32", 1)):
        plan = {"digit_bits": 8, "mode": rs.RS_MODE_MSD, "key_kind": code}
        ko, _ = rs.sort(to_dev(keys), plan=plan)
        vals = np.arange(keys.size, dtype=np.uint32)
        ko2, vo2, _ = rs.sort_pairs(to_dev(keys), to_dev(vals), plan=plan)
        torch.cuda.synchronize()
        rs.rs_check_device_error()
        assert np.array_equal(to_host_u32(ko), oracle.sort_keys(keys, kind))
        wk, wv = oracle.sort_pairs(keys, vals, kind)
        assert np.array_equal(to_host_u32(ko2), wk) and np.array_equal(to_host_u32(vo2), wv)


def test_msd_skewed_top_byte(rs):
    """All keys share the top byte: a few buckets hold everything and go
    through the tiled passes."""
    import torch
    n = 300_000
    keys = (synth.uniform31(n, 1) & np.uint32(0x00FFFFFF)) | np.uint32(0x7A000000)
    ko, _ = rs.sort(to_dev(keys), plan={"mode": rs.RS_MODE_MSD})
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    assert np.array_equal(to_host_u32(ko), oracle.sort_keys(keys))


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_segmented_unaligned_views(rs, shift):
    """Key and value arrays that start 4, 8 or 12 bytes past a 16-byte
    boundary (every kernel of the pipeline reads them through unaligned
    views)."""
    import torch
    sizes = [20_000, 3, 70_001, 16_385, 40_000]
    n = int(sum(sizes))
    keys = synth.uniform31(n, 90 + shift)
    vals = np.arange(n, dtype=np.uint32)
    pad = np.zeros(shift, np.uint32)
    dk = to_dev(np.concatenate([pad, keys]))[shift:]
    dv = to_dev(np.concatenate([pad, vals]))[shift:]
    offs = np.zeros(len(sizes) + 1, np.uint64)
    offs[1:] = np.cumsum(sizes)
    ko, vo, po = rs.sort_segmented(dk, dv, offs)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv, _ = oracle.sort_segmented(keys, vals, offs, 64)
    assert np.array_equal(to_host_u32(ko), wk)
    assert np.array_equal(to_host_u32(vo), wv)
