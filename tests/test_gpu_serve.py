"""The continuous-batching server: each request's result is the same alone
and in the mix (tolerance 0: bit for bit), and equals the oracle's."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _requests(count, seed, rate, lo=1 << 10, hi=1 << 18):
    from paper_cs_0004013_gb300.serve import Request
    out = []
    for q in synth.serving_requests(count, seed, rate_per_s=rate, lo=lo, hi=hi):
        keys = synth.uniform31(q["n"], q["seed"])
        vals = np.arange(q["n"], dtype=np.uint32) if q["pairs"] else None
        out.append(Request.make(q["id"], q["arrival_s"], keys, vals))
    return out


@pytest.mark.parametrize("realtime", [True, False])
def test_results_identical_alone_and_in_the_mix(realtime):
    import torch
    import paper_cs_0004013_gb300 as rs
    from paper_cs_0004013_gb300.serve import SortServer, latency_stats
    reqs = _requests(60, 11, rate=2000.0)
    srv = SortServer(slots=3, streams=3, mem_budget=1 << 30)
    srv.run(reqs, realtime=realtime)
    rs.rs_check_device_error()
    assert len({r.batch for r in reqs}) > 1  # several batches were formed
    for r in reqs:
        got_k, got_v = r.result()
        keys = r.keys.numpy().view(np.uint32)
        dk = r.keys.cuda()
        if r.pairs:
            ko, vo, _ = rs.sort_pairs(dk, r.vals.cuda())  # the same request alone
            torch.cuda.synchronize()
            assert np.array_equal(got_k, ko.cpu().numpy().view(np.uint32)), r.id
            assert np.array_equal(got_v, vo.cpu().numpy().view(np.uint32)), r.id
            wk, wv = oracle.sort_pairs(keys, r.vals.numpy().view(np.uint32))
            assert np.array_equal(got_v, wv)
        else:
            ko, _ = rs.sort(dk)
            torch.cuda.synchronize()
            assert np.array_equal(got_k, ko.cpu().numpy().view(np.uint32)), r.id
            wk = oracle.sort_keys(keys)
        assert np.array_equal(got_k, wk)
    st = latency_stats(reqs)
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_memory_budget_limits_batches():
    """A budget smaller than two requests forces one batch at a time."""
    import paper_cs_0004013_gb300 as rs
    from paper_cs_0004013_gb300.serve import SortServer
    reqs = _requests(12, 12, rate=1e6, lo=1 << 16, hi=1 << 17)
    srv = SortServer(slots=4, streams=2, mem_budget=4 << 20)
    srv.run(reqs, realtime=False)
    rs.rs_check_device_error()
    for r in reqs:
        assert np.array_equal(r.result()[0], oracle.sort_keys(r.keys.numpy().view(np.uint32)))


@pytest.mark.parametrize("realtime", [True, False])
def test_direct_and_batched_requests_mixed(realtime):
    """Requests at or above direct_min_keys are sorted on their own through
    the host-buffer entry point, the rest in segmented batches: every result
    equals the oracle's, whichever way it went."""
    import paper_cs_0004013_gb300 as rs
    from paper_cs_0004013_gb300.serve import SortServer
    reqs = _requests(40, 13, rate=5000.0, lo=1 << 12, hi=1 << 19)
    srv = SortServer(slots=4, streams=3, mem_budget=1 << 30, direct_min_keys=1 << 16)
    srv.run(reqs, realtime=realtime)
    rs.rs_check_device_error()
    big = [r for r in reqs if r.n >= 1 << 16]
    small = [r for r in reqs if r.n < 1 << 16]
    assert big and small
    batches = {}
    for r in reqs:
        batches.setdefault(r.batch, []).append(r)
    for r in big:
        assert batches[r.batch] == [r]  # alone in its batch
    for r in reqs:
        got_k, got_v = r.result()
        keys = r.keys.numpy().view(np.uint32)
        if r.pairs:
            wk, wv = oracle.sort_pairs(keys, r.vals.numpy().view(np.uint32))
            assert np.array_equal(got_v, wv), r.id
        else:
            wk = oracle.sort_keys(keys)
        assert np.array_equal(got_k, wk), r.id


def test_device_error_marks_requests_failed():
    """An error raised on the device while batches run (here the bounded-wait
    self-test, which sets the error word without a fault) is not served as a
    result: the batch that sees it, and every batch in flight with it, are
    marked failed; the run after that is clean."""
    import torch
    import paper_cs_0004013_gb300 as rs
    from paper_cs_0004013_gb300.serve import SortServer, latency_stats
    rs.rs_check_device_error()
    temp = torch.empty(4096, dtype=torch.uint8, device="cuda")
    rs.rs_selftest_wait_timeout(temp)
    torch.cuda.synchronize()
    reqs = _requests(10, 13, rate=1e6)
    srv = SortServer(slots=2, streams=2, mem_budget=1 << 30)
    srv.run(reqs, realtime=False)
    assert srv.failed >= 1
    assert srv.failed == sum(r.error is not None for r in reqs)
    assert all("TIMEOUT" in r.error for r in reqs if r.error is not None)
    rs.rs_check_device_error()  # taken by the server: the word is clear
    reqs2 = _requests(10, 14, rate=1e6)
    srv2 = SortServer(slots=2, streams=2, mem_budget=1 << 30)
    srv2.run(reqs2, realtime=False)
    assert srv2.failed == 0 and all(r.error is None for r in reqs2)
    for r in reqs2:
        got_k, _ = r.result()
        assert np.array_equal(got_k, oracle.sort_keys(r.keys.numpy().view(np.uint32)))
    assert latency_stats(reqs2)["p50_ms"] > 0
