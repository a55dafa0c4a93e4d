"""Host threads sharing the library: each thread sorts on its own stream
with its own temp (keys, pairs, 64-bit keys, merges, tracing switched on by
one of them), and every result equals the oracle's.  Checks the library's
per-device state, its tracing records and its thread-local error messages
under concurrent callers."""
import threading

import numpy as np
import pytest

import oracle
import synth
from tests._gpu import to_dev, to_host_u32

pytestmark = pytest.mark.gpu


def test_concurrent_callers():
    import torch
    import paper_cs_0004013_gb300 as rs
    errors = []
    results = {}

    def worker(i):
        try:
            stream = torch.cuda.Stream()
            n = 100_000 + 977 * i
            keys = synth.uniform31(n, 300 + i)
            with torch.cuda.stream(stream):
                for rep in range(3):
                    if i % 4 == 0:
                        out, _ = rs.sort(to_dev(keys), stream=stream)
                        stream.synchronize()
                        ok = np.array_equal(to_host_u32(out), oracle.sort_keys(keys))
                    elif i % 4 == 1:
                        vals = np.arange(n, dtype=np.uint32)
                        ko, vo, _ = rs.sort_pairs(to_dev(keys), to_dev(vals), stream=stream)
                        stream.synchronize()
                        wk, wv = oracle.sort_pairs(keys, vals)
                        ok = np.array_equal(to_host_u32(ko), wk) and np.array_equal(to_host_u32(vo), wv)
                    elif i % 4 == 2:
                        k64 = synth.splitmix64(400 + i, n)
                        d = torch.from_numpy(k64.view(np.int64).copy()).cuda()
                        out, _ = rs.sort64(d, stream=stream)
                        stream.synchronize()
                        ok = np.array_equal(out.cpu().numpy().view(np.uint64), oracle.sort_keys(k64, "u64"))
                    else:
                        rs.rs_trace_enable(rep % 2 == 0)
                        a, b = oracle.sort_keys(keys), oracle.sort_keys(keys[::-1].copy())
                        out, _, _ = rs.merge(to_dev(a), to_dev(b), stream=stream)
                        stream.synchronize()
                        ok = np.array_equal(to_host_u32(out), oracle.merge(a, b)[0])
                    # a bad call on this thread: its message stays on this thread
                    with pytest.raises(rs.RsError):
                        rs.rs_sort_u32(None, None, 10, plan={"key_kind": 9})
                    assert "key_kind" in rs.rs_last_error()
                    results[(i, rep)] = ok
        except Exception as e:  # reported below
            errors.append((i, repr(e)))

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    rs.rs_trace_enable(False)
    rs.rs_trace_read()
    rs.rs_check_device_error()
    assert not errors, errors
    assert len(results) == 24 and all(results.values()), results
