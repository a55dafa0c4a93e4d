"""The single-launch sort (automatic plan, 16,385 keys up to the resident-tile
limit): one cooperative launch does the histogram, the scans and every pass.
Bit-exact against the oracle, with the trace showing that it ran."""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu import to_dev, to_host_u32

pytestmark = pytest.mark.gpu

TILE = 384 * 24        # the large tile shape
SMALL = 384 * 12       # the smallest tile shape (taken while its tiles number at most one per SM)


@pytest.fixture(scope="module")
def rs():
    import paper_cs_0004013_gb300 as r
    return r


def _run(rs, keys, pairs, kind="u32"):
    import torch
    plan = None if kind == "u32" else {"key_kind": {"i32": 1, "f32": 2}[kind]}
    vals = np.arange(keys.size, dtype=np.uint32)
    rs.rs_trace_read()
    rs.rs_trace_enable(True)
    if pairs:
        ko, vo, offs = rs.sort_pairs(to_dev(keys), to_dev(vals), plan=plan)
    else:
        ko, offs = rs.sort(to_dev(keys), plan=plan)
    torch.cuda.synchronize()
    rs.rs_trace_enable(False)
    tr = rs.rs_trace_read()
    rs.rs_check_device_error()
    if pairs:
        wk, wv = oracle.sort_pairs(keys, vals, kind)
        assert np.array_equal(to_host_u32(vo), wv)
    else:
        wk = oracle.sort_keys(keys, kind)
    assert np.array_equal(to_host_u32(ko), wk)
    assert np.array_equal(offs, oracle.partition_offsets(keys.size, 64))
    return tr


@pytest.mark.parametrize("n", [16385, 4 * SMALL - 1, 4 * SMALL, 4 * SMALL + 1, 2 * TILE - 1, 2 * TILE, 2 * TILE + 1,
                               7 * TILE + 5, 1 << 20, (1 << 21) + 77])
@pytest.mark.parametrize("pairs", [False, True])
def test_sizes(rs, n, pairs):
    keys = synth.uniform31(n, n) | (synth.uniform31(n, n + 3) << np.uint32(1))
    tr = _run(rs, keys, pairs)
    assert tr.get("fused_sort", {}).get("launches") == 1
    assert "onesweep_r8" not in tr and "upfront_hist" not in tr


@pytest.mark.parametrize("dist", sorted(synth.DISTRIBUTIONS))
def test_distributions(rs, dist):
    keys = synth.DISTRIBUTIONS[dist](1 << 20, synth.CONFIG_SEED + 1)
    _run(rs, keys, False)
    _run(rs, keys, True)


@pytest.mark.parametrize("kind", ["zeros", "equal", "low_byte_only", "high_byte_only", "two", "max"])
def test_skipped_digits(rs, kind):
    """Digits with one bucket holding every key are not distributed; every
    digit skipped still copies the keys (stably) into the output."""
    n = 3 * TILE + 311
    u = synth.uniform31(n, 42)
    keys = {"zeros": np.zeros(n, np.uint32), "equal": np.full(n, 0x5A5A5A5A, np.uint32),
            "low_byte_only": (u & np.uint32(0xFF)).astype(np.uint32),
            "high_byte_only": (u & np.uint32(0xFF000000)).astype(np.uint32),
            "two": np.where(u & 1, np.uint32(0xFFFFFFFF), np.uint32(0)).astype(np.uint32),
            "max": np.full(n, 0xFFFFFFFF, np.uint32)}[kind]
    _run(rs, keys, False)
    _run(rs, keys, True)


@pytest.mark.parametrize("kind", ["i32", "f32"])
def test_key_kinds(rs, kind):
    rng = np.random.default_rng(9)
    keys = rng.integers(0, 1 << 32, 300_001, dtype=np.uint64).astype(np.uint32)
    _run(rs, keys, False, kind)
    _run(rs, keys, True, kind)


def test_large_sizes_use_the_pipeline(rs):
    """Above the resident-tile limit the automatic plan goes back to the
    pipeline of launches."""
    n = 1 << 23
    tr = _run(rs, synth.uniform31(n, 1), False)
    assert "fused_sort" not in tr and tr.get("onesweep_r8", {}).get("launches") == 4


@pytest.mark.parametrize("pairs", [False, True])
def test_shape_switch_points(rs, pairs):
    """The tile shape is the smallest whose tiles number at most one per SM
    (384 x 12, then 384 x 18), else 384 x 24 while its tiles all fit; above
    that the pipeline of launches runs.  Sizes on both sides of each switch,
    derived from the SM count, with ragged last tiles."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for n in (sms * 384 * 12 - 7, sms * 384 * 12 + 1, sms * 384 * 18 - 3, sms * 384 * 18 + 1,
              2 * sms * TILE, 2 * sms * TILE + 1):
        keys = synth.uniform31(n, n)
        tr = _run(rs, keys, pairs)
        fused = tr.get("fused_sort", {}).get("launches") == 1
        assert fused or "onesweep_r8" in tr
        if n <= sms * TILE:
            assert fused
