"""Failure detection on the GPU without a fault: a bounded wait that runs
out reports RS_ERR_TIMEOUT through the device error word, and the context
stays usable for the next sort."""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu import to_dev, to_host_u32

pytestmark = pytest.mark.gpu


def test_lookback_wait_gives_up_and_reports():
    import torch
    import paper_cs_0004013_gb300 as rs
    rs.rs_check_device_error()  # start clean
    temp = torch.empty(4096, dtype=torch.uint8, device="cuda")
    rs.rs_selftest_wait_timeout(temp)
    with pytest.raises(rs.RsError) as e:
        rs.rs_check_device_error()
    assert e.value.status == 4  # RS_ERR_TIMEOUT
    rs.rs_check_device_error()  # the word was cleared by the read
    # the context still works
    keys = synth.uniform31(100_000, 3)
    out, _ = rs.sort(to_dev(keys))
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    assert np.array_equal(to_host_u32(out), oracle.sort_keys(keys))


def test_selftest_rejects_small_temp():
    import torch
    import paper_cs_0004013_gb300 as rs
    temp = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(rs.RsError):
        rs.rs_selftest_wait_timeout(temp)


def test_peek_sees_the_word_without_clearing_it():
    """rs_peek_device_error_async copies the word after the stream's work
    and leaves it set; the take then reports and clears it, and a later
    peek reads zero."""
    import torch
    import paper_cs_0004013_gb300 as rs
    rs.rs_check_device_error()  # start clean
    word = torch.full((1,), -1, dtype=torch.int32).pin_memory()
    s = torch.cuda.current_stream()
    rs.rs_peek_device_error_async(word, s)
    s.synchronize()
    assert int(word[0]) == 0
    temp = torch.empty(4096, dtype=torch.uint8, device="cuda")
    rs.rs_selftest_wait_timeout(temp)
    rs.rs_peek_device_error_async(word, s)
    s.synchronize()
    assert int(word[0]) & 1  # bit 0: a bounded wait gave up
    rs.rs_peek_device_error_async(word, s)  # peeking does not clear
    s.synchronize()
    assert int(word[0]) & 1
    with pytest.raises(rs.RsError) as e:
        rs.rs_check_device_error()
    assert e.value.status == 4
    word[0] = -1
    rs.rs_peek_device_error_async(word, s)
    s.synchronize()
    assert int(word[0]) == 0
    with pytest.raises(ValueError):
        rs.rs_peek_device_error_async(torch.zeros(1, dtype=torch.int32, device="cuda"), s)
