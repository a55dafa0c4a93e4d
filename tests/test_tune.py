"""The plan autotuner: candidates, caching, and (on a GPU) that its choice
sorts correctly."""
import math

import numpy as np
import pytest

from paper_cs_0004013_gb300 import tune


def test_size_class_and_candidates():
    assert tune.size_class(1) == 1 and tune.size_class(1000) == 1024 and tune.size_class(1024) == 1024
    c = tune.candidate_plans(1 << 20, pairs=False)
    assert {p["digit_bits"] for p in c} == {8, 11}
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
