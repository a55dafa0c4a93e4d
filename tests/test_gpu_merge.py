"""Parity of the stable merge of sorted runs (rs_merge_u32) with the oracle:
bit-exact keys, payloads (an element of the first run before an equal one
of the second) and partition offsets; empty and ragged runs; every key kind."""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu import to_dev, to_host_u32

pytestmark = pytest.mark.gpu

KIND = {"u32": 0, "i32": 1, "f32": 2}
TILE = 5888  # outputs per default merge tile (keys)


@pytest.fixture(scope="module")
def rs():
    import paper_cs_0004013_gb300 as r
    return r


def _run(seed, n, kind, distinct=None):
    w = synth.splitmix64(seed, (n + 1) // 2).view(np.uint32)[:n].copy()
    if distinct:  # few distinct words: long runs of equal keys across both inputs
        w = w % np.uint32(distinct) * np.uint32(0x01010101)
    return oracle.sort_keys(w, kind)


def _check(rs, a, b, kind, pairs=True):
    import torch
    va = np.arange(a.size, dtype=np.uint32)
    vb = np.arange(a.size, a.size + b.size, dtype=np.uint32)
    ko, vo, offs = rs.merge(to_dev(a), to_dev(b), to_dev(va) if pairs else None, to_dev(vb) if pairs else None,
                            plan={"key_kind": KIND[kind]})
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv = oracle.merge(a, b, va, vb, kind)
    assert np.array_equal(to_host_u32(ko), wk)
    if pairs:
        assert np.array_equal(to_host_u32(vo), wv)
    assert np.array_equal(offs, oracle.partition_offsets(a.size + b.size, 64))


@pytest.mark.parametrize("kind", ["u32", "i32", "f32"])
@pytest.mark.parametrize("sizes", [(0, 0), (0, 5), (5, 0), (1, 1), (1000, 3), (TILE - 1, TILE + 1),
                                   (100_003, 200_001), (1 << 20, 1 << 20)])
def test_sizes(rs, kind, sizes):
    na, nb = sizes
    _check(rs, _run(na + 1, na, kind), _run(nb + 2, nb, kind), kind)


@pytest.mark.parametrize("kind", ["u32", "f32"])
@pytest.mark.parametrize("distinct", [1, 3, 300])
def test_equal_keys_across_runs(rs, kind, distinct):
    """Ties between the runs: every element of the first run comes first."""
    _check(rs, _run(5, 150_001, kind, distinct), _run(6, 70_007, kind, distinct), kind)


def test_disjoint_ranges(rs):
    """One run entirely below the other, in both orders (the merge path runs
    along an edge of the grid)."""
    lo = np.arange(0, 50_000, dtype=np.uint32)
    hi = np.arange(1 << 30, (1 << 30) + 70_000, dtype=np.uint32)
    _check(rs, lo, hi, "u32")
    _check(rs, hi, lo, "u32")


def test_keys_only(rs):
    _check(rs, _run(8, 123_457, "u32"), _run(9, 99_999, "u32"), "u32", pairs=False)


def test_unsorted_runs_stay_in_bounds(rs):
    """Runs that are not sorted: the order is unspecified, but nothing is
    read or written out of bounds; a tile whose path is inconsistent is
    reported through the device error word."""
    import torch
    a = to_dev(synth.uniform31(100_000, 10))
    b = to_dev(synth.uniform31(60_000, 11))
    out, _, _ = rs.merge(a, b)
    torch.cuda.synchronize()
    try:
        rs.rs_check_device_error()
    except rs.RsError:
        pass  # the inconsistent tiles were skipped and reported
    assert out.numel() == 160_000


@pytest.mark.parametrize("tile", [1, 2, 3, 4])
@pytest.mark.parametrize("pairs", [False, True])
def test_tile_shapes(rs, tile, pairs):
    import torch
    a, b = _run(12, 50_001, "u32", 700), _run(13, 33_333, "u32", 700)
    va = np.arange(a.size, dtype=np.uint32)
    vb = np.arange(a.size, a.size + b.size, dtype=np.uint32)
    ko, vo, _ = rs.merge(to_dev(a), to_dev(b), to_dev(va) if pairs else None, to_dev(vb) if pairs else None,
                         plan={"tile": tile})
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv = oracle.merge(a, b, va, vb, "u32")
    assert np.array_equal(to_host_u32(ko), wk)
    if pairs:
        assert np.array_equal(to_host_u32(vo), wv)
