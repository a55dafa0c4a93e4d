"""The serving workload at its full size (40 requests of 2^16..2^26 keys,
half key+payload, the request stream bench.py serves), closed loop through
the continuous-batching server: every keys-only result equals the oracle's
sort, and every key+payload result is pinned by properties that determine it
(ascending keys; payloads = input positions, each exactly once, each carrying
its own key; equal keys with increasing payloads)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_full_serving_workload():
    import torch
    import paper_cs_0004013_gb300 as rs
    from paper_cs_0004013_gb300.serve import Request, SortServer
    reqs = []
    for q in synth.serving_requests(40, synth.CONFIG_SEED + 5, rate_per_s=1e9):
        k = synth.uniform31(q["n"], q["seed"])
        v = np.arange(q["n"], dtype=np.uint32) if q["pairs"] else None
        reqs.append(Request.make(q["id"], q["arrival_s"], k, v))
    srv = SortServer(slots=4, streams=4, mem_budget=24 << 30)
    srv.run(reqs, realtime=False)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    assert any(r.pairs for r in reqs) and any(not r.pairs for r in reqs)
    for r in reqs:
        inp = r.keys.numpy().view(np.uint32)
        got_k, got_v = r.result()
        if not r.pairs:
            assert np.array_equal(got_k, oracle.sort_keys(inp)), r.id
            continue
        assert np.all(got_k[1:] >= got_k[:-1]), r.id
        assert np.array_equal(inp[got_v], got_k), r.id
        seen = np.zeros(r.n, dtype=bool)
        seen[got_v] = True
        assert seen.all(), r.id
        eq = got_k[1:] == got_k[:-1]
        assert np.all(got_v[1:][eq] > got_v[:-1][eq]), r.id
