"""The selection of Sec. 4.2.1 on the GPU against the oracle: the sorted
sample buckets, the problem-cell count and the decision are integers and
must match exactly, for every workload distribution, key kinds, the
paper's parameters and edge sizes."""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu import to_dev, to_host_u32

pytestmark = pytest.mark.gpu

KIND = {"u32": 0, "i32": 1, "f32": 2}


@pytest.fixture(scope="module")
def rs():
    import paper_cs_0004013_gb300 as r
    return r


def _check(rs, keys, kind="u32", bits=13, sample=1000, cells=64, max_problem=2):
    import torch
    d = to_dev(keys)
    s = min(sample, keys.size)
    db = torch.zeros(max(s, 1), dtype=torch.int32, device="cuda")
    got = rs.rs_sample_overlap(d, keys.size, KIND[kind], bits, sample, cells, max_problem, db)
    wb, wp, wc = oracle.choose_plan(keys, kind, bits=bits, sample=sample, cells=cells, max_problem=max_problem)
    assert got["sample"] == wb.size
    assert np.array_equal(to_host_u32(db)[: wb.size], wb)
    assert got["problem_cells"] == wp and got["clustered"] == wc
    return got


@pytest.mark.parametrize("dist", sorted(synth.DISTRIBUTIONS))
def test_workload_distributions(rs, dist):
    keys = synth.DISTRIBUTIONS[dist](1 << 20, synth.CONFIG_SEED + 7)
    _check(rs, keys)


def test_clustered_and_uniform_decisions(rs):
    assert not _check(rs, synth.uniform31(1 << 22, 3))["clustered"]
    assert _check(rs, synth.tight_clusters(1 << 22, 3))["clustered"]
    assert _check(rs, np.full(3000, 9, np.uint32))["problem_cells"] == 63


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 999, 1000, 1001, 123457])
def test_edge_sizes(rs, n):
    _check(rs, synth.gauss_mix(n, n))


@pytest.mark.parametrize("kind", ["i32", "f32"])
def test_key_kinds(rs, kind):
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 1 << 32, 50000, dtype=np.uint64).astype(np.uint32)
    keys[::7] = keys[0]
    _check(rs, keys, kind)


@pytest.mark.parametrize("params", [dict(bits=2, sample=8, cells=4), dict(bits=32, sample=1024, cells=1024),
                                    dict(bits=11, sample=500, cells=7, max_problem=0)])
def test_other_parameters(rs, params):
    _check(rs, synth.few_distinct(20000, 11), **params)


def test_choose_plan_vetoes_bucketing_on_clustered_data(rs):
    """rs_choose_plan keeps an MSD plan for uniform keys and turns it into
    LSD for clustered ones; an LSD plan is kept either way."""
    msd = {"digit_bits": 8, "mode": rs.RS_MODE_MSD}
    plan, st = rs.rs_choose_plan(to_dev(synth.uniform31(1 << 20, 1)), 1 << 20, msd)
    assert plan["mode"] == rs.RS_MODE_MSD and not st["clustered"]
    plan, st = rs.rs_choose_plan(to_dev(synth.tight_clusters(1 << 20, 1)), 1 << 20, msd)
    assert plan["mode"] == rs.RS_MODE_LSD and st["clustered"]
    plan, st = rs.rs_choose_plan(to_dev(synth.tight_clusters(1 << 20, 1)), 1 << 20, {"mode": rs.RS_MODE_LSD})
    assert plan["mode"] == rs.RS_MODE_LSD


def test_rejects_bad_parameters(rs):
    d = to_dev(synth.uniform31(100, 1))
    for kw in (dict(sample=0), dict(sample=1025), dict(cells=0), dict(bits=0), dict(bits=33), dict(key_kind=9)):
        with pytest.raises(rs.RsError):
            rs.rs_sample_overlap(d, 100, **kw)
