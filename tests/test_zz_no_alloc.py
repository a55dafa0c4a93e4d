"""rs_sort_u32_noalloc, the sort for callers that cannot allocate device memory
(a host program that owns every allocation, a latency-critical path that
cannot afford cudaMalloc, code that must not run out of memory mid-run): its
scratch is a fixed array inside the library, so the caller passes only the
keys, the output and the offsets array.

The output must equal the regular entry point's (rs_sort_u32, whose scratch
the caller allocates) bit for bit, on calls made back to back, because every
call reuses the same array and must not see the previous call's leftovers.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import gc

import numpy as np
import pytest

import synth
from tests._gpu import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_cs_0004013_gb300 as r
    return r


def test_noalloc_matches_regular_entry_point_on_back_to_back_calls(rs):
    import torch
    cases = [(rs.RS_NOALLOC_MAX_KEYS, 1), (123_457, 2), (rs.RS_NOALLOC_MAX_KEYS, 3), (1, 4), (0, 5)]
    for n, salt in cases:
        keys = synth.uniform31(n, 9000 + salt) | (synth.uniform31(n, 9100 + salt) << np.uint32(1))
        d = to_dev(keys.astype(np.uint32))
        want, want_offs = rs.sort(d, num_parts=64)  # regular entry point, caller-allocated scratch
        for _ in range(2):  # two calls in a row on the shared scratch
            got = torch.full_like(d, -1)
            offs = rs.rs_sort_u32_noalloc(d, got, n, 64)
            torch.cuda.synchronize()
            rs.rs_check_device_error()
            assert torch.equal(got, want), n
            assert np.array_equal(offs, want_offs), n


def test_noalloc_calls_allocate_no_device_memory(rs):
    """The property the entry point exists for: once the first call on the
    device has set it up, further calls change neither PyTorch's allocation
    count nor the device's free memory."""
    import torch
    n = rs.RS_NOALLOC_MAX_KEYS
    d = to_dev(synth.uniform31(n, 9200))
    got = torch.empty_like(d)
    rs.rs_sort_u32_noalloc(d, got, 0, 64)  # set-up only
    rs.rs_sort_u32_noalloc(d, got, n, 64)  # warm-up: every kernel the sort uses is loaded
    torch.cuda.synchronize()
    gc.collect()
    torch.cuda.reset_peak_memory_stats()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    for _ in range(4):
        rs.rs_sort_u32_noalloc(d, got, n, 64)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    # no allocation through PyTorch (its peak stays where it was) and none
    # from the driver (free device memory unchanged)
    assert torch.cuda.max_memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_more_keys_than_its_scratch_holds(rs):
    with pytest.raises(rs.RsError) as e:
        rs.rs_sort_u32_noalloc(None, None, rs.RS_NOALLOC_MAX_KEYS + 1, 64)
    assert e.value.status == 1  # RS_ERR_INVALID
    assert "no-alloc limit" in rs.rs_last_error()
