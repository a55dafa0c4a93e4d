"""Parity with the oracle for signed and binary32 keys (rs_plan.key_kind):
every plan and entry point, bit-exact, on words drawn over all 32-bit
patterns (NaNs of both signs, both zeros, infinities, denormals) and on
inputs that exercise digit skipping."""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu import to_dev, to_host_u32, to_host_u64

pytestmark = pytest.mark.gpu

TILE = 12288
KIND = {"i32": 1, "f32": 2}
SPECIAL = np.array([0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0xFFC00000, 0x7F800001,
                    0xFFFFFFFF, 0x00000001, 0x80000001, 0x7F7FFFFF, 0xFF7FFFFF, 0x7FFFFFFF, 0x3F800000,
                    0xBF800000], np.uint32)


@pytest.fixture(scope="module")
def rs():
    import paper_cs_0004013_gb300 as r
    return r


def _words(n, seed):
    w = synth.splitmix64(seed, (n + 1) // 2).view(np.uint32)[:n].copy()
    if n >= SPECIAL.size * 4:  # special values, each several times, at seeded places
        pos = synth.splitmix64(seed + 1, SPECIAL.size * 4) % np.uint64(n)
        w[pos.astype(np.int64)] = np.tile(SPECIAL, 4)
    return w


def _check(rs, keys, kind, plan=None, pairs=False):
    import torch
    plan = dict(plan or {}, key_kind=KIND[kind])
    d = to_dev(keys)
    if pairs:
        vals = np.arange(keys.size, dtype=np.uint32)
        ko, vo, offs = rs.sort_pairs(d, to_dev(vals), plan=plan)
    else:
        ko, offs = rs.sort(d, plan=plan)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    if pairs:
        wk, wv = oracle.sort_pairs(keys, vals, kind)
        assert np.array_equal(to_host_u32(vo), wv)
    else:
        wk = oracle.sort_keys(keys, kind)
    assert np.array_equal(to_host_u32(ko), wk)
    assert np.array_equal(offs, oracle.partition_offsets(keys.size, 64))
    assert np.array_equal(to_host_u32(d), keys), "input modified"


@pytest.mark.parametrize("kind", ["i32", "f32"])
@pytest.mark.parametrize("n", [1, 2, 1000, 3 * TILE + 5, 1 << 20])
@pytest.mark.parametrize("pairs", [False, True])
def test_default_plan(rs, kind, n, pairs):
    _check(rs, _words(n, 11 + n), kind, pairs=pairs)


@pytest.mark.parametrize("kind", ["i32", "f32"])
@pytest.mark.parametrize("plan", [{"digit_bits": 8, "mode": 1, "tile": 1}, {"digit_bits": 8, "mode": 1, "tile": 3},
                                  {"digit_bits": 8, "mode": 1, "tile": 6}, {"digit_bits": 11, "mode": 1},
                                  {"digit_bits": 8, "mode": 2}])
def test_plans(rs, kind, plan):
    keys = _words(300_001, 29)
    _check(rs, keys, kind, plan)
    _check(rs, keys, kind, plan, pairs=True)


@pytest.mark.parametrize("kind", ["i32", "f32"])
def test_skipped_digits_and_all_equal(rs, kind):
    n = 100_003
    # small negative integers: after the order map the top three bytes agree
    small_neg = (-(synth.uniform31(n, 3) % np.uint32(200)).astype(np.int64) - 1).astype(np.int32).view(np.uint32)
    _check(rs, small_neg, kind, pairs=True)
    # every key the same word: every digit skipped, the pass is a copy
    for w in (0xBF800000, 0x80000000, 0x7FC00000):
        _check(rs, np.full(n, w, np.uint32), kind, pairs=True)
    # one bucket of -0 and +0 (f32: distinct words, -0 first)
    _check(rs, np.where(synth.uniform31(n, 4) & np.uint32(1), np.uint32(0x80000000), np.uint32(0)), kind,
           pairs=True)


@pytest.mark.parametrize("kind", ["i32", "f32"])
def test_segmented(rs, kind):
    import torch
    sizes = [0, 1, 5, 4095, 4097, 16385, 3 * TILE + 7, 70_001, 2]
    n = int(sum(sizes))
    keys = _words(n, 31)
    vals = np.arange(n, dtype=np.uint32)
    offs = np.zeros(len(sizes) + 1, np.uint64)
    offs[1:] = np.cumsum(sizes)
    ko, vo, po = rs.sort_segmented(to_dev(keys), to_dev(vals), offs, plan={"key_kind": KIND[kind]})
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    wk, wv, wp = oracle.sort_segmented(keys, vals, offs, 64, kind)
    assert np.array_equal(to_host_u32(ko), wk)
    assert np.array_equal(to_host_u32(vo), wv)
    assert np.array_equal(to_host_u64(po).reshape(len(sizes), 65), wp)


@pytest.mark.parametrize("kind", ["i32", "f32"])
def test_host_entry(rs, kind):
    import torch
    n = 200_001
    keys = _words(n, 37)
    hk = torch.from_numpy(keys.view(np.int32).copy()).pin_memory()
    ho = torch.empty_like(hk).pin_memory()
    plan = {"key_kind": KIND[kind]}
    temp = torch.empty(rs.rs_sort_u32_host(None, None, None, None, n, plan=plan), dtype=torch.uint8,
                       device="cuda")
    rs.rs_sort_u32_host(hk, None, ho, None, n, 64, plan, temp)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    assert np.array_equal(ho.numpy().view(np.uint32), oracle.sort_keys(keys, kind))


def test_float_tensor_in_float_tensor_out(rs):
    """A float32 tensor sorted as binary32 keys comes back as float32 values
    in ascending order (numpy's order off NaN and signed zeros)."""
    import torch
    x = torch.from_numpy(np.linspace(-1e30, 1e30, 100_001, dtype=np.float32)[::-1].copy()).cuda()
    out, _ = rs.sort(x, plan={"key_kind": rs.RS_KEY_F32})
    torch.cuda.synchronize()
    assert out.dtype == torch.float32
    assert np.array_equal(out.cpu().numpy(), np.sort(x.cpu().numpy()))


def test_unknown_key_kind_is_rejected(rs):
    with pytest.raises(rs.RsError):
        rs.rs_sort_u32(None, None, 100, plan={"key_kind": 7})
