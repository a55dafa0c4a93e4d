"""The C-ABI library loads and exports every entry point the header declares;
argument checks that need no GPU.  (No compute calls: no GPU here.)"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsort.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("rs_sort_u32", "rs_sort_u32_pairs", "rs_sort_u32_segmented", "rs_last_error",
                 "rs_check_device_error", "rs_digit_histograms", "rs_radix_pass", "rs_version"):
        assert want in names


def test_library_exports_every_declared_symbol():
    import paper_cs_0004013_gb300 as r
    dll = ctypes.CDLL(r.LIBRARY_PATH)
    missing = [n for n in declared_functions() if not hasattr(dll, n)]
    assert not missing, missing


def test_version_and_no_error_initially():
    import paper_cs_0004013_gb300 as r
    assert r.rs_version() >= 10000
    assert r.rs_last_error() == ""


def test_temp_queries_grow_with_n_and_payload():
    import paper_cs_0004013_gb300 as r
    a = r.rs_sort_u32(None, None, 1 << 20)
    b = r.rs_sort_u32(None, None, 1 << 22)
    c = r.rs_sort_u32_pairs(None, None, None, None, 1 << 22)
    assert 0 < a < b < c
    assert r.rs_sort_u32(None, None, 0) > 0
    # the alternate key buffer dominates: at least 4 bytes per key
    assert b >= 4 * (1 << 22)
    assert c >= 8 * (1 << 22)
    for bits in (8, 11):
        assert r.rs_sort_u32(None, None, 1 << 20, plan={"digit_bits": bits}) > 0


@pytest.mark.parametrize("call", ["n_too_big", "bad_bits", "bad_parts", "msd_pending", "bad_tile", "bad_kind",
                                  "bad_kind_segmented"])
def test_invalid_arguments(call):
    import paper_cs_0004013_gb300 as r
    with pytest.raises(r.RsError) as e:
        if call == "n_too_big":
            r.rs_sort_u32(None, None, 1 << 32)
        elif call == "bad_bits":
            r.rs_sort_u32(None, None, 100, plan={"digit_bits": 9})
        elif call == "bad_parts":
            r.rs_sort_u32(None, None, 10, num_parts=0)
        elif call == "msd_pending":
            r.rs_sort_u32(None, None, 100, plan={"mode": 99})
        elif call == "bad_kind":
            r.rs_sort_u32_pairs(None, None, None, None, 100, plan={"key_kind": 3})
        elif call == "bad_kind_segmented":
            import numpy as np
            r.rs_sort_u32_segmented(None, None, None, None, None, np.array([0, 100], np.uint64), 1, 100,
                                    plan={"key_kind": 9})
        else:
            r.rs_sort_u32(None, None, 100, plan={"tile": 42})
    assert r.rs_last_error() != ""


def test_temp_too_small_and_misaligned_are_rejected():
    import paper_cs_0004013_gb300 as r
    need = r.rs_sort_u32(None, None, 1000)
    sz = ctypes.c_size_t(need - 1)
    st = r.lib.rs_sort_u32(ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 24), 1000, 64, None, None,
                           ctypes.c_void_p(1 << 28), ctypes.byref(sz), None)
    assert st == 2  # RS_ERR_TEMP_TOO_SMALL
    sz = ctypes.c_size_t(need)
    st = r.lib.rs_sort_u32(ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 24), 1000, 64, None, None,
                           ctypes.c_void_p((1 << 28) + 16), ctypes.byref(sz), None)
    assert st == 1  # misaligned temp


def test_overlapping_buffers_are_rejected():
    import paper_cs_0004013_gb300 as r
    need = r.rs_sort_u32(None, None, 1000)
    sz = ctypes.c_size_t(need)
    # keys_out overlaps keys_in
    st = r.lib.rs_sort_u32(ctypes.c_void_p(1 << 20), ctypes.c_void_p((1 << 20) + 400), 1000, 64, None, None,
                           ctypes.c_void_p(1 << 28), ctypes.byref(sz), None)
    assert st == 1 and "overlap" in r.rs_last_error()
    # keys_out inside temp
    st = r.lib.rs_sort_u32(ctypes.c_void_p(1 << 20), ctypes.c_void_p((1 << 28) + 256), 1000, 64, None, None,
                           ctypes.c_void_p(1 << 28), ctypes.byref(sz), None)
    assert st == 1


def test_partition_offsets_host_path_needs_no_gpu():
    """n = 0 returns the offsets without touching the device."""
    import numpy as np
    import paper_cs_0004013_gb300 as r
    need = r.rs_sort_u32(None, None, 0)
    offs = np.ones(65, dtype=np.uint64)
    sz = ctypes.c_size_t(need)
    st = r.lib.rs_sort_u32(None, None, 0, 64, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), None,
                           ctypes.c_void_p(1 << 28), ctypes.byref(sz), None)
    assert st == 0 and not offs.any()


def test_host_entry_sizes_and_checks():
    """rs_sort_u32_host: its temp is the device sort's plus device copies of
    the arrays; argument errors are caught before any copy."""
    import numpy as np
    import paper_cs_0004013_gb300 as r
    n = 1000
    slot = (4 * n + 255) // 256 * 256
    assert r.rs_sort_u32_host(None, None, None, None, n) == r.rs_sort_u32(None, None, n) + 2 * slot
    assert (r.rs_sort_u32_host(None, 1, None, 2, n)
            == r.rs_sort_u32_pairs(None, None, None, None, n) + 4 * slot)
    for args in ((None, 1, None, None), (None, None, None, 2)):  # values on one side only
        with pytest.raises(r.RsError):
            r.rs_sort_u32_host(*args, n)
    with pytest.raises(r.RsError):
        r.rs_sort_u32_host(None, None, None, None, n, num_parts=0)
    need = r.rs_sort_u32_host(None, None, None, None, n)
    keys = np.zeros(2 * n, dtype=np.uint32)
    base = keys.ctypes.data
    sz = ctypes.c_size_t(need)
    st = r.lib.rs_sort_u32_host(base, None, base + 400, None, n, 64, None, None, ctypes.c_void_p(1 << 28),
                                ctypes.byref(sz), None)
    assert st == 1 and "overlap" in r.rs_last_error()
    sz = ctypes.c_size_t(need - 1)
    st = r.lib.rs_sort_u32_host(base, None, base + 4 * n, None, n, 64, None, None, ctypes.c_void_p(1 << 28),
                                ctypes.byref(sz), None)
    assert st == 2
    offs = np.ones(65, dtype=np.uint64)
    sz = ctypes.c_size_t(r.rs_sort_u32_host(None, None, None, None, 0))
    st = r.lib.rs_sort_u32_host(None, None, None, None, 0, 64, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                None, ctypes.c_void_p(1 << 28), ctypes.byref(sz), None)
    assert st == 0 and not offs.any()


def test_wide_temp_queries():
    """Temp of the 64-bit sorts: the default tile shape reads and writes
    interleaved words (four key-word planes); other shapes split the keys
    (six); 64-bit values add one index plane to the 32-bit-value layout."""
    import paper_cs_0004013_gb300 as r
    n = 1 << 22
    k = r.rs_sort_u64(None, None, n)
    kp = r.rs_sort_u64_pairs(None, None, None, None, n)
    kp64 = r.rs_sort_u64_pairs64(None, None, None, None, n)
    assert 16 * n <= k < kp < kp64
    assert kp64 - kp >= 4 * n
    # another key+payload shape (tile 6): split planes, two more per key word
    assert r.rs_sort_u64(None, None, n, plan={"tile": 6}) >= k + 8 * n
    with pytest.raises(r.RsError):
        r.rs_sort_u64_pairs64(None, None, None, None, n, plan={"mode": 2})  # MSD is not offered for 64-bit keys
    # against the same plan (8-bit LSD on 512 x 16 tiles, the shape with the
    # two-payload-word kernels that the 64-bit-value sort runs)
    v64 = r.rs_sort_u32_pairs64(None, None, None, None, n)
    same = {"digit_bits": 8, "mode": r.RS_MODE_LSD, "tile": 1}
    assert v64 >= r.rs_sort_u32_pairs(None, None, None, None, n, plan=same) + 12 * n


def test_wide_entries_reject_bad_buffers_before_any_launch():
    """64-bit keys and values: misaligned or overlapping buffers are refused
    on the host (fake device addresses; nothing is launched)."""
    import paper_cs_0004013_gb300 as r
    n = 1000
    P = ctypes.c_void_p
    need = r.rs_sort_u64_pairs64(None, None, None, None, n)
    sz = ctypes.c_size_t(need)
    keys_in, keys_out, vals_in, vals_out, temp = 1 << 20, 1 << 21, 1 << 22, 1 << 23, 1 << 28
    # values misaligned for 8-byte words
    st = r.lib.rs_sort_u64_pairs64(P(keys_in), P(vals_in + 4), P(keys_out), P(vals_out), n, 64, None, None,
                                   P(temp), ctypes.byref(sz), None)
    assert st == 1 and "aligned" in r.rs_last_error()
    # vals_out overlapping keys_out
    st = r.lib.rs_sort_u64_pairs64(P(keys_in), P(vals_in), P(keys_out), P(keys_out + 4000), n, 64, None, None,
                                   P(temp), ctypes.byref(sz), None)
    assert st == 1 and "overlap" in r.rs_last_error()
    # temp one byte short
    short = ctypes.c_size_t(need - 1)
    st = r.lib.rs_sort_u64_pairs64(P(keys_in), P(vals_in), P(keys_out), P(vals_out), n, 64, None, None,
                                   P(temp), ctypes.byref(short), None)
    assert st == 2
    # 32-bit keys with 64-bit values: the same alignment rule
    need = r.rs_sort_u32_pairs64(None, None, None, None, n)
    sz = ctypes.c_size_t(need)
    st = r.lib.rs_sort_u32_pairs64(P(keys_in), P(vals_in + 4), P(keys_out), P(vals_out), n, 64, None, None,
                                   P(temp), ctypes.byref(sz), None)
    assert st == 1 and "aligned" in r.rs_last_error()
    # 64-bit keys must be 8-byte aligned
    need = r.rs_sort_u64(None, None, n)
    sz = ctypes.c_size_t(need)
    st = r.lib.rs_sort_u64(P(keys_in + 4), P(keys_out), n, 64, None, None, P(temp), ctypes.byref(sz), None)
    assert st == 1 and "aligned" in r.rs_last_error()
