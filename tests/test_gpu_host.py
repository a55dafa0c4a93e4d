"""Parity of the host-buffer entry point (rs_sort_u32_host) with the oracle:
host arrays in, host arrays out, bit-exact; calls on two streams whose
copies and sorts overlap stay independent."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_cs_0004013_gb300 as r
    return r


def _host(a: np.ndarray, pinned: bool):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.int32).copy())
    return t.pin_memory() if pinned else t


def _run(rs, keys, vals=None, pinned=True, plan=None, stream=None):
    import torch
    n = keys.size
    hk = _host(keys, pinned)
    hv = _host(vals, pinned) if vals is not None else None
    ok = torch.zeros_like(hk).pin_memory() if pinned else torch.zeros_like(hk)
    ov = None if vals is None else (torch.zeros_like(hv).pin_memory() if pinned else torch.zeros_like(hv))
    nb = rs.rs_sort_u32_host(None, hv, None, ov, n, plan=plan)
    temp = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
    offs = rs.rs_sort_u32_host(hk, hv, ok, ov, n, 64, plan, temp, stream)
    return hk, ok, ov, offs, temp


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("n", [0, 1, 1000, 300_001])
def test_host_keys(rs, n, pinned):
    import torch
    keys = synth.uniform31(n, 21)
    hk, ok, _, offs, _ = _run(rs, keys, pinned=pinned)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    assert np.array_equal(ok.numpy().view(np.uint32), oracle.sort_keys(keys))
    assert np.array_equal(offs, oracle.partition_offsets(n, 64))
    assert np.array_equal(hk.numpy().view(np.uint32), keys), "input modified"


@pytest.mark.parametrize("dist", ["uniform", "few_distinct", "tight_clusters"])
def test_host_pairs(rs, dist):
    import torch
    n = 123_457
    keys = synth.DISTRIBUTIONS[dist](n, 5)
    vals = np.arange(n, dtype=np.uint32)
    _, ok, ov, offs, _ = _run(rs, keys, vals)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    sk, sv = oracle.sort_pairs(keys, vals)
    assert np.array_equal(ok.numpy().view(np.uint32), sk)
    assert np.array_equal(ov.numpy().view(np.uint32), sv)
    assert np.array_equal(offs, oracle.partition_offsets(n, 64))


def test_host_two_streams_overlap(rs):
    """Four sorts alternating over two streams (each call with its own temp):
    every output is that of its own input."""
    import torch
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    runs = []
    for i in range(4):
        keys = synth.uniform31((1 << 20) + 7 * i, 40 + i)
        runs.append((keys, _run(rs, keys, stream=streams[i % 2])))
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    for keys, (_, ok, _, _, _) in runs:
        assert np.array_equal(ok.numpy().view(np.uint32), oracle.sort_keys(keys))


def test_host_plans(rs):
    """The host path runs the same device plans (LSD 8/11-bit, MSD)."""
    import torch
    keys = synth.tight_clusters(200_003, 9)
    for plan in ({"digit_bits": 8, "mode": 1}, {"digit_bits": 11, "mode": 1}, {"digit_bits": 8, "mode": 2}):
        _, ok, _, _, _ = _run(rs, keys, plan=plan)
        torch.cuda.synchronize()
        rs.rs_check_device_error()
        assert np.array_equal(ok.numpy().view(np.uint32), oracle.sort_keys(keys)), plan
