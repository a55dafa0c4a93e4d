"""Plans installed for a size class (by the autotuner or the caller) are the
ones calls without a plan run, and they stay bit-exact against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from paper_cs_0004013_gb300 import tune
from tests._gpu import to_dev, to_host_u32, to_host_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_cs_0004013_gb300 as r
    return r


def _segments(seed, count=60, lo=2000, hi=16000):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi, count)
    offs = np.zeros(count + 1, np.uint64)
    offs[1:] = np.cumsum(sizes)
    return offs


def test_installed_plain_plan_is_the_one_that_runs(rs):
    """An 11-bit plan installed for the 2^20 class: a call without a plan
    runs 11-bit passes (trace), keys and pairs match the oracle; removing
    the entry brings back the compiled default (8-bit passes, in one launch)."""
    import torch
    n = (1 << 20) - 3  # class 20
    keys = synth.gauss_mix(n, 41)
    vals = np.arange(n, dtype=np.uint32)
    for entry in (rs.RS_ENTRY_SORT_U32, rs.RS_ENTRY_SORT_U32_PAIRS):
        rs.rs_set_default_plan(entry, 20, {"digit_bits": 11, "mode": 1, "tile": 2})
    try:
        rs.rs_trace_read()
        rs.rs_trace_enable(True)
        out, offs = rs.sort(to_dev(keys))
        ko, vo, _ = rs.sort_pairs(to_dev(keys), to_dev(vals))
        torch.cuda.synchronize()
        rs.rs_trace_enable(False)
        tr = rs.rs_trace_read()
        rs.rs_check_device_error()
        assert tr.get("onesweep_r11", {}).get("launches", 0) >= 6 and "onesweep_r8" not in tr
        assert np.array_equal(to_host_u32(out), oracle.sort_keys(keys))
        assert np.array_equal(offs, oracle.partition_offsets(n, 64))
        wk, wv = oracle.sort_pairs(keys, vals)
        assert np.array_equal(to_host_u32(ko), wk) and np.array_equal(to_host_u32(vo), wv)
    finally:
        for entry in (rs.RS_ENTRY_SORT_U32, rs.RS_ENTRY_SORT_U32_PAIRS):
            rs.rs_set_default_plan(entry, 20, None)
    rs.rs_trace_enable(True)
    out, _ = rs.sort(to_dev(keys))
    torch.cuda.synchronize()
    rs.rs_trace_enable(False)
    tr = rs.rs_trace_read()
    # the compiled default at this size: the single-launch sort (8-bit passes)
    assert "onesweep_r11" not in tr and ("fused_sort" in tr or "onesweep_r8" in tr)
    assert np.array_equal(to_host_u32(out), oracle.sort_keys(keys))


@pytest.mark.parametrize("pairs", [False, True])
def test_installed_segmented_plan_is_the_one_that_runs(rs, pairs):
    """A segmented plan installed for the batch's class changes the launch
    layout (the temp size of the 512 x 16 shape differs from the default's)
    and the output stays the oracle's."""
    import torch
    offs = _segments(5)
    S, n = offs.size - 1, int(offs[-1])
    cls = tune.size_log2(-(-n // S))
    entry = rs.RS_ENTRY_SEGMENTED_PAIRS if pairs else rs.RS_ENTRY_SEGMENTED
    keys = synth.uniform31(n, 42)
    vals = np.arange(n, dtype=np.uint32)
    dv = to_dev(vals) if pairs else None
    plan = {"digit_bits": 8, "mode": rs.RS_MODE_LSD, "tile": 1}
    default_bytes = rs.rs_sort_u32_segmented(None, dv, None, dv, None, offs, S, n, 64)
    explicit_bytes = rs.rs_sort_u32_segmented(None, dv, None, dv, None, offs, S, n, 64, plan=plan)
    assert explicit_bytes != default_bytes
    rs.rs_set_default_plan(entry, cls, plan)
    try:
        assert rs.rs_sort_u32_segmented(None, dv, None, dv, None, offs, S, n, 64) == explicit_bytes
        ko, vo, po = rs.sort_segmented(to_dev(keys), dv, offs)
        torch.cuda.synchronize()
        rs.rs_check_device_error()
    finally:
        rs.rs_set_default_plan(entry, cls, None)
    wk, wv, wp = oracle.sort_segmented(keys, vals if pairs else None, offs, 64)
    assert np.array_equal(to_host_u32(ko), wk)
    if pairs:
        assert np.array_equal(to_host_u32(vo), wv)
    assert np.array_equal(to_host_u64(po).reshape(S, 65), wp)


@pytest.mark.parametrize("plan", [{"tile": 1, "mode": 1}, {"tile": 1, "mode": 2}, {"tile": 2, "mode": 1},
                                  {"tile": 2, "mode": 2}, {"tile": 3, "mode": 1}, {"tile": 3, "mode": 2}])
def test_every_segmented_candidate_matches_the_oracle(rs, plan):
    import torch
    offs = np.concatenate([[0], np.cumsum([0, 1, 4095, 4097, 16384, 16385, 30000, 3, 70000])]).astype(np.uint64)
    S, n = offs.size - 1, int(offs[-1])
    keys = synth.few_distinct(n, 17)
    vals = np.arange(n, dtype=np.uint32)
    ko, vo, po = rs.sort_segmented(to_dev(keys), to_dev(vals), offs, plan=dict(plan, digit_bits=8))
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv, wp = oracle.sort_segmented(keys, vals, offs, 64)
    assert np.array_equal(to_host_u32(ko), wk) and np.array_equal(to_host_u32(vo), wv)
    assert np.array_equal(to_host_u64(po).reshape(S, 65), wp)


def test_tuner_end_to_end_on_a_batch(rs, tmp_path):
    """The tuner times the segmented candidates on a batch, installs the
    winner, and a call without a plan then runs it, bit-exact."""
    import torch
    offs = _segments(9, count=40)
    S, n = offs.size - 1, int(offs[-1])
    keys = synth.uniform31(n, 43)
    vals = np.arange(n, dtype=np.uint32)
    dk, dv = to_dev(keys), to_dev(vals)
    t = tune.Tuner(cache_path=str(tmp_path / "plans.json"), reps=1)
    best = t.best_segmented_plan(offs, pairs=True, keys=dk, vals=dv)
    assert best in tune.segmented_candidates(True)
    assert t.install() >= 1
    cls = tune.size_log2(-(-n // S))
    try:
        assert rs.rs_get_default_plan(rs.RS_ENTRY_SEGMENTED_PAIRS, cls) == best
        ko, vo, _ = rs.sort_segmented(dk, dv, offs)
        torch.cuda.synchronize()
        rs.rs_check_device_error()
    finally:
        rs.rs_set_default_plan(rs.RS_ENTRY_SEGMENTED_PAIRS, cls, None)
    wk, wv, _ = oracle.sort_segmented(keys, vals, offs, 64)
    assert np.array_equal(to_host_u32(ko), wk) and np.array_equal(to_host_u32(vo), wv)
