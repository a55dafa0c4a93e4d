"""The largest inputs: n above 2^30 - 2^16, where a 32-bit chained-scan
status word (30-bit count field) can no longer hold a running count, so the
passes switch to 64-bit status words.  The oracle cannot sort 2^30 keys in
seconds, so the output is checked on properties that hold at any size
(ascending order, the same multiset of top-16-bit buckets as the input, for
pairs a stable permutation) and, exactly, on sampled positions whose values
the oracle computes one by one: the sampled position's bucket of the input
is gathered and sorted on its own."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

N = (1 << 30) + 12345  # past the 32-bit status limit, with a ragged last tile
CHUNK = 1 << 26
BUCKET_SHIFT = 15      # 31-bit keys: 65,536 buckets of the top 16 bits


def _need_gpu_bytes(pairs: bool) -> int:
    words = 4 if pairs else 2           # inputs and outputs
    alt = 2 if pairs else 1             # the alternate buffers
    status = (N // 8192 + 2) * 256 * 8  # 64-bit status rows of one pass
    return N * 4 * (words + alt) + status + (1 << 30)


def _keys(seed: int):
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    return torch.randint(0, (1 << 31) - 1, (N,), generator=g, device="cuda", dtype=torch.int32)


def _bucket_hist(a: np.ndarray) -> np.ndarray:
    h = np.zeros(1 << 16, np.int64)
    for s in range(0, a.size, CHUNK):
        h += np.bincount(a[s:s + CHUNK] >> BUCKET_SHIFT, minlength=1 << 16)
    return h


def _check_sorted(out: np.ndarray) -> None:
    for s in range(0, out.size - 1, CHUNK):
        e = min(s + CHUNK, out.size - 1)
        assert np.all(out[s + 1:e + 1] >= out[s:e]), f"not ascending in [{s}, {e}]"


def _sampled_positions(n: int) -> np.ndarray:
    rng = np.random.default_rng(7)
    return np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1], rng.integers(0, n, 6)]))


def _expected_at(inp: np.ndarray, hist: np.ndarray, pos: np.ndarray) -> np.ndarray:
    """The oracle's value at each sampled output position: the position's
    bucket (from the input's cumulative bucket counts), that bucket's keys
    gathered from the input and sorted by the oracle, then indexed."""
    cum = np.cumsum(hist)
    bkt = np.searchsorted(cum, pos, side="right")
    want = {int(b): [] for b in bkt}
    for s in range(0, inp.size, CHUNK):
        c = inp[s:s + CHUNK]
        cb = c >> BUCKET_SHIFT
        for b in want:
            want[b].append(c[cb == b])
    out = []
    for p, b in zip(pos, bkt):
        keys = oracle.sort_keys(np.concatenate(want[int(b)]))
        before = int(cum[b - 1]) if b > 0 else 0
        out.append(keys[int(p) - before])
    return np.array(out, dtype=np.uint32)


def test_wide_status_keys():
    import torch
    import paper_cs_0004013_gb300 as rs
    free, _ = torch.cuda.mem_get_info()
    if free < _need_gpu_bytes(False):
        pytest.skip("not enough free device memory")
    d = _keys(2024)
    out, offs = rs.sort(d)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    inp = d.cpu().numpy().view(np.uint32)
    res = out.cpu().numpy().view(np.uint32)
    del d, out
    assert np.array_equal(offs, oracle.partition_offsets(N, 64))
    _check_sorted(res)
    hist = _bucket_hist(inp)
    assert np.array_equal(hist, _bucket_hist(res))
    pos = _sampled_positions(N)
    assert np.array_equal(res[pos], _expected_at(inp, hist, pos))


def test_wide_status_pairs_stable():
    import torch
    import paper_cs_0004013_gb300 as rs
    free, _ = torch.cuda.mem_get_info()
    if free < _need_gpu_bytes(True):
        pytest.skip("not enough free device memory")
    # few distinct keys: long runs of equal keys exercise stability
    dk = _keys(77) & ((1 << 31) - (1 << 20))
    dv = torch.arange(N, dtype=torch.int32, device="cuda")
    ko, vo, offs = rs.sort_pairs(dk, dv)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    inp = dk.cpu().numpy().view(np.uint32)
    keys = ko.cpu().numpy().view(np.uint32)
    vals = vo.cpu().numpy().view(np.uint32)
    del dk, dv, ko, vo
    assert np.array_equal(offs, oracle.partition_offsets(N, 64))
    _check_sorted(keys)
    seen = np.zeros(N, dtype=bool)
    for s in range(0, N, CHUNK):
        v = vals[s:s + CHUNK]
        assert np.array_equal(inp[v], keys[s:s + CHUNK]), "payload does not point at its key"
        seen[v] = True
    assert seen.all(), "payloads are not a permutation"
    for s in range(0, N - 1, CHUNK):
        e = min(s + CHUNK, N - 1)
        eq = keys[s + 1:e + 1] == keys[s:e]
        assert np.all(vals[s + 1:e + 1][eq] > vals[s:e][eq]), "equal keys lost their input order"
