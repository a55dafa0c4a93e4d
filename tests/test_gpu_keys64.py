"""Parity of the 64-bit key sort (rs_sort_u64) with the oracle, bit-exact:
unsigned, signed and binary64 keys over all 64-bit patterns, digits skipped
in either word, every key+payload tile shape."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TILE = 8192  # keys per tile of the default key+payload kernel
KIND = {"u64": 0, "i64": 1, "f64": 2}
SPECIAL = np.array([0, 1 << 63, 0x7FF0000000000000, 0xFFF0000000000000, 0x7FF8000000000000, 0xFFF8000000000000,
                    0x7FF0000000000001, 2**64 - 1, 1, (1 << 63) + 1, 0x7FEFFFFFFFFFFFFF, 0xFFEFFFFFFFFFFFFF,
                    2**63 - 1, 0x3FF0000000000000, 0xBFF0000000000000, 0x00000000FFFFFFFF, 0xFFFFFFFF00000000],
                   np.uint64)


@pytest.fixture(scope="module")
def rs():
    import paper_cs_0004013_gb300 as r
    return r


def _words(n, seed):
    w = synth.splitmix64(seed, n)
    if n >= SPECIAL.size * 4:
        pos = (synth.splitmix64(seed + 1, SPECIAL.size * 4) % np.uint64(n)).astype(np.int64)
        w[pos] = np.tile(SPECIAL, 4)
    return w


def _check(rs, keys, kind, plan=None):
    import torch
    d = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    out, offs = rs.sort64(d, plan=dict(plan or {}, key_kind=KIND[kind]))
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    assert np.array_equal(out.cpu().numpy().view(np.uint64), oracle.sort_keys(keys, kind))
    assert np.array_equal(offs, oracle.partition_offsets(keys.size, 64))
    assert np.array_equal(d.cpu().numpy().view(np.uint64), keys), "input modified"


@pytest.mark.parametrize("kind", ["u64", "i64", "f64"])
@pytest.mark.parametrize("n", [1, 2, 1000, 3 * TILE + 5, 1 << 20])
def test_kinds_and_sizes(rs, kind, n):
    _check(rs, _words(n, 50 + n), kind)


@pytest.mark.parametrize("kind", ["u64", "i64", "f64"])
def test_skipped_digits(rs, kind):
    n = 200_003
    r = synth.splitmix64(61, n)
    _check(rs, r & np.uint64(0xFFFFFFFF), kind)                 # high word constant: its four digits skip
    _check(rs, r & np.uint64(0xFFFFFFFF00000000), kind)         # low word constant
    _check(rs, (r & np.uint64(0xFF)) | np.uint64(0xC000000000000000), kind)  # seven digits constant
    _check(rs, np.full(n, 0xBFF0000000000000, np.uint64), kind)  # every digit skipped: a copy


@pytest.mark.parametrize("tile", list(range(1, 9)))
def test_tile_shapes(rs, tile):
    plan = {"tile": tile}
    try:
        rs.rs_sort_u64(None, None, 1000, plan=plan)
    except rs.RsError:
        pytest.skip(f"no key+payload kernel for tile shape {tile}")
    _check(rs, _words(5 * TILE + 777, 71), "u64", plan)


def test_empty_and_offsets_only(rs):
    import torch
    d = torch.empty(0, dtype=torch.int64, device="cuda")
    out, offs = rs.sort64(d)
    assert out.numel() == 0 and not offs.any()


def test_float64_tensor(rs):
    import torch
    x = torch.from_numpy(np.linspace(-1e300, 1e300, 100_001)[::-1].copy()).cuda()
    out, _ = rs.sort64(x, plan={"key_kind": rs.RS_KEY_F32})
    torch.cuda.synchronize()
    assert out.dtype == torch.float64
    assert np.array_equal(out.cpu().numpy(), np.sort(x.cpu().numpy()))


def _check_pairs(rs, keys, kind, plan=None):
    import torch
    vals = np.arange(keys.size, dtype=np.uint32)
    dk = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    ko, vo, offs = rs.sort64_pairs(dk, dv, plan=dict(plan or {}, key_kind=KIND[kind]))
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv = oracle.sort_pairs(keys, vals, kind)
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), wk)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), wv)
    assert np.array_equal(offs, oracle.partition_offsets(keys.size, 64))


@pytest.mark.parametrize("kind", ["u64", "i64", "f64"])
@pytest.mark.parametrize("n", [1, 1000, 3 * TILE + 5, 1 << 20])
def test_pairs(rs, kind, n):
    _check_pairs(rs, _words(n, 80 + n), kind)


@pytest.mark.parametrize("kind", ["u64", "f64"])
def test_pairs_stable_and_skipped(rs, kind):
    n = 300_007
    r = synth.splitmix64(83, n)
    _check_pairs(rs, r % np.uint64(97) * np.uint64(0x0101010101010101), kind)  # few distinct keys
    _check_pairs(rs, r & np.uint64(0xFFFF00000000), kind)                    # six digits constant
    _check_pairs(rs, np.full(n, 0xC000000000000000, np.uint64), kind)        # every digit skipped


@pytest.mark.parametrize("kind", ["u32", "i32", "f32"])
@pytest.mark.parametrize("n", [1, 1000, 3 * TILE + 5, 1 << 20])
def test_u32_keys_u64_values(rs, kind, n):
    """32-bit keys carrying 64-bit values (rs_sort_u32_pairs64): stable."""
    import torch
    keys = synth.splitmix64(90 + n, (n + 1) // 2).view(np.uint32)[:n].copy()
    keys[::3] = keys[0]  # many equal keys
    vals = synth.splitmix64(91 + n, n) ^ np.arange(n, dtype=np.uint64)
    dk = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int64).copy()).cuda()
    ko, vo, offs = rs.sort_pairs64(dk, dv, plan={"key_kind": {"u32": 0, "i32": 1, "f32": 2}[kind]})
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv = oracle.sort_pairs(keys, vals, kind)
    assert np.array_equal(ko.cpu().numpy().view(np.uint32), wk)
    assert np.array_equal(vo.cpu().numpy().view(np.uint64), wv)
    assert np.array_equal(offs, oracle.partition_offsets(n, 64))


@pytest.mark.parametrize("tile", [0, 6])
def test_keys_off_16_byte_boundary(rs, tile):
    """Keys and values that start 8 bytes past a 16-byte boundary, odd
    lengths: the interleaved reads take a head and a tail element apart
    (tile 6 takes the split word planes instead)."""
    import torch
    n = 3 * TILE + 7
    keys = _words(n + 1, 95)
    d = torch.from_numpy(keys.view(np.int64).copy()).cuda()[1:]
    assert d.data_ptr() % 16 == 8
    out, _ = rs.sort64(d, plan={"tile": tile, "key_kind": KIND["f64"]})
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    assert np.array_equal(out.cpu().numpy().view(np.uint64), oracle.sort_keys(keys[1:], "f64"))
    k32 = synth.uniform31(n, 96)
    dv = torch.from_numpy(keys.view(np.int64).copy()).cuda()[1:]
    ko, vo, _ = rs.sort_pairs64(torch.from_numpy(k32.view(np.int32)).cuda(), dv)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv = oracle.sort_pairs(k32, keys[1:], "u32")
    assert np.array_equal(ko.cpu().numpy().view(np.uint32), wk)
    assert np.array_equal(vo.cpu().numpy().view(np.uint64), wv)


def _check_pairs64(rs, keys, kind, plan=None, vals=None):
    import torch
    n = keys.size
    if vals is None:
        vals = synth.splitmix64(77 + n, n) ^ np.arange(n, dtype=np.uint64)  # distinct, every bit pattern
    dk = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int64).copy()).cuda()
    ko, vo, offs = rs.sort64_pairs(dk, dv, plan=dict(plan or {}, key_kind=KIND[kind]))
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv = oracle.sort_pairs(keys, vals, kind)
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), wk)
    assert np.array_equal(vo.cpu().numpy().view(np.uint64), wv)
    assert np.array_equal(offs, oracle.partition_offsets(n, 64))
    assert np.array_equal(dv.cpu().numpy().view(np.uint64), vals), "values modified"


@pytest.mark.parametrize("kind", ["u64", "i64", "f64"])
@pytest.mark.parametrize("n", [1, 2, 1000, 3 * TILE + 5, 1 << 20])
def test_u64_keys_u64_values(rs, kind, n):
    """64-bit keys carrying 64-bit values (rs_sort_u64_pairs64): the passes
    carry an input index, the last one gathers the values; stable."""
    _check_pairs64(rs, _words(n, 100 + n), kind)


@pytest.mark.parametrize("kind", ["u64", "f64"])
def test_u64_values_stable_and_skipped(rs, kind):
    n = 300_007
    r = synth.splitmix64(101, n)
    _check_pairs64(rs, r % np.uint64(97) * np.uint64(0x0101010101010101), kind)  # few distinct keys
    _check_pairs64(rs, r & np.uint64(0xFFFF00000000), kind)                    # six digits constant
    _check_pairs64(rs, r & np.uint64(0xFF), kind)                              # seven digits constant
    # every digit skipped: the one pass both makes the indices and gathers
    _check_pairs64(rs, np.full(n, 0xC000000000000000, np.uint64), kind)


def test_u64_values_unaligned_and_persistent(rs):
    import torch
    n = 2 * TILE + 3
    keys = _words(n, 102)
    vals = synth.splitmix64(103, n + 1)
    dk = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int64).copy()).cuda()[1:]  # 8 bytes past a 16-byte boundary
    ko, vo, _ = rs.sort64_pairs(dk, dv)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv = oracle.sort_pairs(keys, vals[1:], "u64")
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), wk)
    assert np.array_equal(vo.cpu().numpy().view(np.uint64), wv)
    for tile in range(1, 14):  # shapes without an interleaved two-payload-word kernel are refused on the host
        try:
            rs.rs_sort_u64_pairs64(None, None, None, None, 1000, plan={"tile": tile})
        except rs.RsError:
            continue
        _check_pairs64(rs, keys, "u64", {"tile": tile})
