"""The plan autotuner: candidates, caching, and (on a GPU) that its choice
sorts correctly."""
import math

import numpy as np
import pytest

from paper_cs_0004013_gb300 import tune


def test_size_class_and_candidates():
    assert tune.size_class(1) == 1 and tune.size_class(1000) == 1024 and tune.size_class(1024) == 1024
    c = tune.candidate_plans(1 << 20, pairs=False)
    assert {p["digit_bits"] for p in c} == {0, 8, 11}
    assert {"digit_bits": 0, "mode": tune.RS_MODE_AUTO, "tile": 0} in c  # the automatic plan competes too
    assert any(p["mode"] == tune.RS_MODE_MSD for p in c)
    assert not any(p["mode"] == tune.RS_MODE_MSD for p in tune.candidate_plans((1 << 30) - 1, True))


def test_picks_fastest_and_caches(tmp_path, monkeypatch):
    t = tune.Tuner(cache_path=str(tmp_path / "plans.json"))
    calls = []

    def fake_time(plan, keys, vals=None):
        calls.append(plan)
        if plan["digit_bits"] == 11:
            return math.inf  # unavailable
        return 10.0 - plan["tile"] if plan["mode"] == tune.RS_MODE_LSD else 50.0

    monkeypatch.setattr(t, "time_plan", fake_time)
    best = t.best_plan(1 << 20, False, keys=object(), gpu="FAKE GPU")
    top = max(p["tile"] for p in tune.candidate_plans(1 << 20, False)
              if p["digit_bits"] == 8 and p["mode"] == tune.RS_MODE_LSD)
    assert best == {"digit_bits": 8, "mode": tune.RS_MODE_LSD, "tile": top}
    n_calls = len(calls)
    again = tune.Tuner(cache_path=str(tmp_path / "plans.json"))
    monkeypatch.setattr(again, "time_plan", fake_time)
    assert again.best_plan(1000 * 1000, False, keys=object(), gpu="FAKE GPU") == best  # same size class, cached
    assert len(calls) == n_calls
    assert again.best_plan(1 << 20, True, keys=object(), gpu="FAKE GPU") == best  # pairs: timed again
    assert len(calls) > n_calls


def test_segmented_candidates_cover_shapes_and_modes():
    c = tune.segmented_candidates(pairs=True)
    assert {(p["tile"], p["mode"]) for p in c} == {(t, m) for t in (1, 2, 3)
                                                   for m in (tune.RS_MODE_MSD, tune.RS_MODE_LSD)}


def test_segmented_pick_uses_mean_segment_size_class(tmp_path, monkeypatch):
    t = tune.Tuner(cache_path=str(tmp_path / "plans.json"))
    calls = []

    def fake_time(plan, keys, vals, h_offs):
        calls.append(plan)
        return 1.0 if (plan["tile"], plan["mode"]) == (1, tune.RS_MODE_LSD) else 2.0

    monkeypatch.setattr(t, "time_segmented", fake_time)
    offs = np.array([0, 3000, 9000, 12000], dtype=np.uint64)  # mean 4000 -> class 12
    best = t.best_segmented_plan(offs, pairs=False, keys=object(), gpu="FAKE GPU")
    assert best == {"digit_bits": 8, "mode": tune.RS_MODE_LSD, "tile": 1}
    assert "FAKE GPU|segmented|12|keys|uniform" in t._load()
    n = len(calls)
    assert t.best_segmented_plan(np.array([0, 4096], dtype=np.uint64), keys=object(), gpu="FAKE GPU") == best
    assert len(calls) == n  # same class: cached


def test_install_hands_cached_winners_to_the_library(tmp_path, monkeypatch):
    """The library's plan table (host-only entry points: no GPU needed)
    receives the cached winners of this GPU and nothing else."""
    import paper_cs_0004013_gb300 as rs
    t = tune.Tuner(cache_path=str(tmp_path / "plans.json"))
    t._load().update({
        "FAKE GPU|plain|20|keys|uniform": {"plan": {"digit_bits": 11, "mode": 1, "tile": 2}},
        "FAKE GPU|segmented|13|pairs|uniform": {"plan": {"digit_bits": 8, "mode": 1, "tile": 1}},
        "FAKE GPU|plain|21|keys|clustered": {"plan": {"digit_bits": 8, "mode": 1, "tile": 3}},
        "OTHER GPU|plain|22|keys|uniform": {"plan": {"digit_bits": 8, "mode": 1, "tile": 3}},
    })
    try:
        assert t.install(gpu="FAKE GPU") == 2
        assert rs.rs_get_default_plan(rs.RS_ENTRY_SORT_U32, 20) == {"digit_bits": 11, "mode": 1, "tile": 2}
        assert rs.rs_get_default_plan(rs.RS_ENTRY_SEGMENTED_PAIRS, 13) == {"digit_bits": 8, "mode": 1, "tile": 1}
        assert rs.rs_get_default_plan(rs.RS_ENTRY_SORT_U32, 21) is None
        assert rs.rs_get_default_plan(rs.RS_ENTRY_SORT_U32, 22) is None
    finally:
        rs.rs_set_default_plan(rs.RS_ENTRY_SORT_U32, 20, None)
        rs.rs_set_default_plan(rs.RS_ENTRY_SEGMENTED_PAIRS, 13, None)
    assert rs.rs_get_default_plan(rs.RS_ENTRY_SORT_U32, 20) is None


def test_default_plan_table_rejects_bad_entries():
    import paper_cs_0004013_gb300 as rs
    for args in ((4, 10, {"digit_bits": 8}), (0, 33, {"digit_bits": 8}), (0, 10, {"digit_bits": 9}),
                 (0, 10, {"mode": 7}), (0, 10, {"key_kind": 1})):
        with pytest.raises(rs.RsError):
            rs.rs_set_default_plan(*args)


@pytest.mark.gpu
def test_tuned_plan_sorts_correctly(tmp_path):
    import torch
    import oracle
    import synth
    import paper_cs_0004013_gb300 as rs
    t = tune.Tuner(cache_path=str(tmp_path / "plans.json"), reps=1)
    plan = t.best_plan(1 << 20, pairs=True)
    keys = synth.uniform31((1 << 20) + 5, 8)
    vals = np.arange(keys.size, dtype=np.uint32)
    ko, vo, _ = rs.sort_pairs(torch.from_numpy(keys.view(np.int32)).cuda(),
                              torch.from_numpy(vals.view(np.int32)).cuda(), plan=plan)
    torch.cuda.synchronize()
    wk, wv = oracle.sort_pairs(keys, vals)
    assert np.array_equal(ko.cpu().numpy().view(np.uint32), wk)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), wv)
