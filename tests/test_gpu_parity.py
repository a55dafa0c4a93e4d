"""Parity of the CUDA path (through the C ABI) with the oracle: bit-exact.

Every step of the method is checked on its own (digit histograms and their
cumulative totals, one stable distribution pass) and as a whole (keys,
pairs with payload = input position, segmented), on the seeded workloads
and on edge cases: empty, one element, ragged tails around the tile size,
all-equal keys, extreme values, digits that are skipped."""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu import to_dev, to_host_u32, to_host_u64

pytestmark = pytest.mark.gpu

TILE = 8192  # keys per tile of the default kernels


@pytest.fixture(scope="module")
def rs():
    import paper_cs_0004013_gb300 as r
    return r


def _sort_check(rs, keys, plan=None, num_parts=64):
    import torch
    d = to_dev(keys)
    out, offs = rs.sort(d, num_parts=num_parts, plan=plan)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    assert np.array_equal(to_host_u32(out), oracle.sort_keys(keys))
    assert np.array_equal(offs, oracle.partition_offsets(keys.size, num_parts))
    assert np.array_equal(to_host_u32(d), keys), "input modified"


def _pairs_check(rs, keys, vals=None, plan=None, num_parts=64):
    import torch
    vals = np.arange(keys.size, dtype=np.uint32) if vals is None else vals
    dk, dv = to_dev(keys), to_dev(vals)
    ko, vo, offs = rs.sort_pairs(dk, dv, num_parts=num_parts, plan=plan)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    sk, sv = oracle.sort_pairs(keys, vals)
    assert np.array_equal(to_host_u32(ko), sk)
    assert np.array_equal(to_host_u32(vo), sv)
    assert np.array_equal(offs, oracle.partition_offsets(keys.size, num_parts))


# ------------------------------------------------------------ single steps
@pytest.mark.parametrize("bits", [8, 11])
@pytest.mark.parametrize("dist", ["uniform", "tight_clusters", "few_distinct", "small"])
@pytest.mark.parametrize("n", [1, 1000, 3 * TILE + 5, 1 << 20])
def test_digit_histograms_and_bases(rs, bits, dist, n):
    import torch
    keys = (synth.uniform31(n, 3) & np.uint32(0x3FF)) if dist == "small" else synth.DISTRIBUTIONS[dist](n, 7)
    plan = oracle.digit_plan(bits)
    nd, B = len(plan), 1 << bits
    h = torch.zeros(nd * B, dtype=torch.int32, device="cuda")
    b = torch.zeros_like(h)
    s = torch.zeros(nd, dtype=torch.int32, device="cuda")
    # an unaligned view of the keys exercises the head/tail path of the kernel
    dk = to_dev(np.concatenate([[np.uint32(7)], keys]))[1:]
    rs.rs_digit_histograms(dk, n, bits, h, b, s)
    torch.cuda.synchronize()
    want_h = oracle.digit_histograms(keys, plan)
    got_h = to_host_u32(h).reshape(nd, B)
    got_b = to_host_u32(b).reshape(nd, B)
    for j, (sh, w) in enumerate(plan):
        assert np.array_equal(got_h[j, : 1 << w], want_h[j]), (j, sh, w)
        assert not got_h[j, 1 << w:].any()
        assert np.array_equal(got_b[j, : 1 << w], oracle.digit_bases(want_h[j]))
    assert list(to_host_u32(s)) == [int(x) for x in oracle.skippable_digits(want_h, n)]


@pytest.mark.parametrize("shift,width", [(0, 8), (8, 8), (24, 8), (0, 11), (11, 11), (22, 10), (3, 5), (31, 1)])
@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("n", [1, 777, 2 * TILE, 5 * TILE + 123])
def test_radix_pass(rs, shift, width, pairs, n):
    import torch
    keys = synth.gauss_mix(n, 11)
    vals = np.arange(n, dtype=np.uint32)
    dk, dv = to_dev(keys), to_dev(vals)
    ko, vo = torch.empty_like(dk), torch.empty_like(dv)
    temp = torch.empty(rs.rs_radix_pass(None, None, None, None, n, shift, width), dtype=torch.uint8,
                       device="cuda")
    rs.rs_radix_pass(dk, dv if pairs else None, ko, vo if pairs else None, n, shift, width, temp)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv = oracle.distribute(keys, vals, shift, width)
    assert np.array_equal(to_host_u32(ko), wk)
    if pairs:
        assert np.array_equal(to_host_u32(vo), wv)


# --------------------------------------------------------------- whole sort
EDGE_N = [0, 1, 2, 3, 63, 64, 65, 1000, TILE - 1, TILE, TILE + 1, 4 * TILE + 17, (1 << 20) + 7]


@pytest.mark.parametrize("n", EDGE_N)
@pytest.mark.parametrize("bits", [8, 11])
def test_sort_edge_sizes(rs, n, bits):
    keys = synth.uniform31(n, 100 + n).astype(np.uint32) | (synth.uniform31(n, 5) << np.uint32(1))
    _sort_check(rs, keys, plan={"digit_bits": bits})
    _pairs_check(rs, keys, plan={"digit_bits": bits})


@pytest.mark.parametrize("kind", ["zeros", "max", "equal", "two", "sorted", "reverse", "topbit", "onebit",
                                  "low_byte_only", "high_byte_only"])
def test_sort_edge_values(rs, kind):
    n = 3 * TILE + 311
    u = synth.uniform31(n, 42)
    keys = {
        "zeros": np.zeros(n, np.uint32),
        "max": np.full(n, 0xFFFFFFFF, np.uint32),
        "equal": np.full(n, 0x5A5A5A5A, np.uint32),
        "two": np.where(u & 1, np.uint32(0xFFFFFFFF), np.uint32(0)).astype(np.uint32),
        "sorted": np.sort(u),
        "reverse": np.sort(u)[::-1].copy(),
        "topbit": (u | np.uint32(1 << 31)).astype(np.uint32),
        "onebit": (np.uint32(1) << (u % np.uint32(32))).astype(np.uint32),
        "low_byte_only": (u & np.uint32(0xFF)).astype(np.uint32),
        "high_byte_only": (u & np.uint32(0xFF000000)).astype(np.uint32),
    }[kind]
    for bits in (8, 11):
        _sort_check(rs, keys, plan={"digit_bits": bits})
        _pairs_check(rs, keys, plan={"digit_bits": bits})


@pytest.mark.parametrize("kind", ["low_digit_mostly_zero", "low_digit_two_values", "runs_of_equal_keys"])
def test_concentrated_digits_multi_launch(rs, kind):
    """Above 2^22 keys (the pipeline of launches with the half-warp-group
    kernel): inputs whose digits leave most lanes of a warp on one digit,
    where the first pass's atomic ranking and the later passes' mask words
    meet the most contention."""
    n = (1 << 22) + 12345
    u = synth.uniform31(n, 7)
    hi = u & np.uint32(0xFFFFFF00)
    keys = {
        "low_digit_mostly_zero": hi | np.where(u % np.uint32(100) == 0, u & np.uint32(0xFF), 0).astype(np.uint32),
        "low_digit_two_values": hi | ((u >> np.uint32(20)) & np.uint32(1)),
        "runs_of_equal_keys": np.repeat(synth.uniform31(n // 1000 + 1, 8), 1000)[:n],
    }[kind].astype(np.uint32)
    _sort_check(rs, keys)
    _pairs_check(rs, keys)


@pytest.mark.parametrize("tile", list(range(1, 9)))
@pytest.mark.parametrize("bits", [8, 11])
def test_tile_shapes(rs, tile, bits):
    """Every registered tile shape (plain and persistent pipelined kernels),
    keys and pairs, LSD mode, on sizes spanning many tiles and a ragged tail."""
    plan = {"digit_bits": bits, "tile": tile, "mode": rs.RS_MODE_LSD}
    try:
        rs.temp_bytes(1000, pairs=False, plan=plan)
    except rs.RsError:
        pytest.skip(f"no tile shape {tile} for {bits}-bit digits")
    try:
        rs.temp_bytes(1000, pairs=True, plan=plan)
        with_pairs = True
    except rs.RsError:  # a keys-only shape
        with_pairs = False
    for n in (5 * TILE + 999, 1 << 20, 37):
        keys = synth.few_distinct(n, 9 + n) if n > 100 else synth.uniform31(n, 1)
        _sort_check(rs, keys, plan=plan)
        if with_pairs:
            _pairs_check(rs, keys, plan=plan)


@pytest.mark.parametrize("dist", sorted(synth.DISTRIBUTIONS))
def test_workload_distributions_small(rs, dist):
    keys = synth.DISTRIBUTIONS[dist](1 << 20, synth.CONFIG_SEED + 3)
    _sort_check(rs, keys)
    _pairs_check(rs, keys)


def test_workload_uniform_2_20_keys(rs):
    """2^20 uniform 31-bit keys, keys only, 64 partitions."""
    _sort_check(rs, synth.config_keys(1))


@pytest.mark.parametrize("num_parts", [1, 7, 64, 1000])
def test_partition_counts(rs, num_parts):
    _sort_check(rs, synth.uniform31(12345, 1), num_parts=num_parts)


# -------------------------------------------------------------- full sizes
def test_full_uniform_2_26_keys_and_pairs(rs):
    keys = synth.config_keys(2)
    _sort_check(rs, keys)
    _pairs_check(rs, keys)


@pytest.mark.parametrize("dist", ["skewed_chunks", "few_distinct", "gauss_mix", "tight_clusters"])
def test_full_distributions_2_26(rs, dist):
    _sort_check(rs, synth.config_keys(3, dist=dist))


# ----------------------------------------------------------------- segmented
@pytest.mark.parametrize("pairs", [False, True])
def test_segmented_mixed_sizes(rs, pairs):
    import torch
    sizes = [0, 1, 5, 0, TILE + 3, 3, 100000, 0, 2, 70000, 1]
    offs = np.zeros(len(sizes) + 1, np.uint64)
    offs[1:] = np.cumsum(sizes)
    n = int(offs[-1])
    keys = synth.gauss_mix(n, 77)
    vals = np.arange(n, dtype=np.uint32)
    dk = to_dev(keys)
    dv = to_dev(vals) if pairs else None
    ko, vo, po = rs.sort_segmented(dk, dv, offs, num_parts=64)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv, wp = oracle.sort_segmented(keys, vals if pairs else None, offs, 64)
    assert np.array_equal(to_host_u32(ko), wk)
    if pairs:
        assert np.array_equal(to_host_u32(vo), wv)
    assert np.array_equal(to_host_u64(po).reshape(len(sizes), 65), wp)
