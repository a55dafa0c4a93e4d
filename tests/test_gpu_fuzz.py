"""Seeded random cases across every plan boundary of the plain sorts: sizes
log-uniform from 1 key to 2^23 (one-block local sort, the single-launch sort
with each of its tile shapes, the pipeline of launches with each default
tile), every workload distribution, key kinds, keys only and with payloads,
bit-exact against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu import to_dev, to_host_u32

pytestmark = pytest.mark.gpu

CASES = 24


@pytest.fixture(scope="module")
def rs():
    import paper_cs_0004013_gb300 as r
    return r


def _case(i):
    rng = np.random.default_rng(0xF022 + i)
    n = int(np.exp(rng.uniform(0.0, np.log(1 << 23))))
    dist = sorted(synth.DISTRIBUTIONS)[int(rng.integers(len(synth.DISTRIBUTIONS)))]
    kind = ("u32", "u32", "i32", "f32")[int(rng.integers(4))]
    pairs = bool(rng.integers(2))
    return n, dist, kind, pairs


@pytest.mark.parametrize("i", range(CASES))
def test_random_case(rs, i):
    import torch
    n, dist, kind, pairs = _case(i)
    keys = synth.DISTRIBUTIONS[dist](n, 1000 + i)
    if kind != "u32":  # every 32-bit pattern of the kind, both signs
        keys = synth.splitmix64(2000 + i, (n + 1) // 2).view(np.uint32)[:n].copy()
    plan = None if kind == "u32" else {"key_kind": {"i32": 1, "f32": 2}[kind]}
    vals = np.arange(n, dtype=np.uint32)
    if pairs:
        ko, vo, offs = rs.sort_pairs(to_dev(keys), to_dev(vals), plan=plan)
    else:
        ko, offs = rs.sort(to_dev(keys), plan=plan)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    if pairs:
        wk, wv = oracle.sort_pairs(keys, vals, kind)
        assert np.array_equal(to_host_u32(vo), wv), (n, dist, kind)
    else:
        wk = oracle.sort_keys(keys, kind)
    assert np.array_equal(to_host_u32(ko), wk), (n, dist, kind, pairs)
    assert np.array_equal(offs, oracle.partition_offsets(n, 64))
