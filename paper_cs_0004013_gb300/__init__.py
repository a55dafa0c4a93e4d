"""Python binding of librsort: a GB300 radix distribution sort of uint32 keys.

Argument marshalling only: every step of the sort runs in the CUDA kernels
of ``librsort.so`` (built in-tree by ``build.py``).  The functions named
``rs_*`` mirror the C entry points of ``include/rsort.h`` one to one and take
torch CUDA tensors (int32 or uint32; only their device pointers are used).
``sort``, ``sort_pairs`` and ``sort_segmented`` are conveniences that also
allocate the outputs and the temp buffer through torch.

There is no fallback: if the library is missing or fails to load, importing
this package raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as LIBRARY_PATH

__all__ = [
    "RsError", "RsPlan", "lib", "LIBRARY_PATH",
    "rs_sort_u32", "rs_sort_u32_pairs", "rs_sort_u32_segmented", "rs_digit_histograms",
    "rs_radix_pass", "rs_last_error", "rs_check_device_error", "rs_peek_device_error_async", "rs_version", "rs_trace_enable",
    "rs_trace_read", "rs_sort_u32_noalloc", "RS_NOALLOC_MAX_KEYS", "rs_selftest_wait_timeout",
    "rs_sort_u32_host", "rs_sort_u64", "sort64", "rs_sort_u64_pairs", "rs_sort_u64_pairs64", "sort64_pairs", "rs_sort_u32_pairs64", "sort_pairs64", "rs_merge_u32", "merge",
    "sort", "sort_pairs", "sort_segmented", "temp_bytes",
    "STATUS_NAMES", "RS_MODE_AUTO", "RS_MODE_LSD", "RS_MODE_MSD", "RS_KEY_U32", "RS_KEY_I32", "RS_KEY_F32",
    "rs_set_default_plan", "rs_get_default_plan", "RS_ENTRY_SORT_U32", "RS_ENTRY_SORT_U32_PAIRS",
    "RS_ENTRY_SEGMENTED", "RS_ENTRY_SEGMENTED_PAIRS", "rs_sample_overlap", "rs_choose_plan",
]

STATUS_NAMES = {0: "RS_OK", 1: "RS_ERR_INVALID", 2: "RS_ERR_TEMP_TOO_SMALL", 3: "RS_ERR_CUDA",
                4: "RS_ERR_TIMEOUT", 5: "RS_ERR_UNSUPPORTED"}
RS_MODE_AUTO, RS_MODE_LSD, RS_MODE_MSD = 0, 1, 2
# key kinds (rs_plan.key_kind): how 32-bit key words are ordered
RS_KEY_U32, RS_KEY_I32, RS_KEY_F32 = 0, 1, 2
RS_NOALLOC_MAX_KEYS = 1 << 20


class RsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class RsTraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("total_ms", ctypes.c_double), ("keys", ctypes.c_double)]


class RsPlan(ctypes.Structure):
    _fields_ = [("digit_bits", ctypes.c_uint32), ("mode", ctypes.c_uint32),
                ("tile", ctypes.c_uint32), ("key_kind", ctypes.c_uint32)]


_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_SZP = ctypes.POINTER(ctypes.c_size_t)
_U64P = ctypes.POINTER(ctypes.c_uint64)
_PLANP = ctypes.POINTER(RsPlan)

_SIGS = {
    "rs_sort_u32": [_P, _P, _U64, _U32, _U64P, _PLANP, _P, _SZP, _P],
    "rs_sort_u32_pairs": [_P, _P, _P, _P, _U64, _U32, _U64P, _PLANP, _P, _SZP, _P],
    "rs_sort_u32_segmented": [_P, _P, _P, _P, _P, _U64P, _U32, _U64, _U32, _P, _PLANP, _P, _SZP, _P],
    "rs_digit_histograms": [_P, _U64, _U32, _P, _P, _P, _P],
    "rs_radix_pass": [_P, _P, _P, _P, _U64, _U32, _U32, _P, _SZP, _P],
    "rs_last_error": [],
    "rs_check_device_error": [_P],
    "rs_peek_device_error_async": [_P, _P],
    "rs_version": [],
    "rs_trace_enable": [ctypes.c_int],
    "rs_sort_u32_host": [_P, _P, _P, _P, _U64, _U32, _U64P, _PLANP, _P, _SZP, _P],
    "rs_sort_u64": [_P, _P, _U64, _U32, _U64P, _PLANP, _P, _SZP, _P],
    "rs_sort_u64_pairs": [_P, _P, _P, _P, _U64, _U32, _U64P, _PLANP, _P, _SZP, _P],
    "rs_sort_u32_pairs64": [_P, _P, _P, _P, _U64, _U32, _U64P, _PLANP, _P, _SZP, _P],
    "rs_sort_u64_pairs64": [_P, _P, _P, _P, _U64, _U32, _U64P, _PLANP, _P, _SZP, _P],
    "rs_merge_u32": [_P, _P, _U64, _P, _P, _U64, _P, _P, _U32, _U64P, _PLANP, _P, _SZP, _P],
    "rs_sort_u32_noalloc": [_P, _P, _U64, _U32, _U64P, _P],
    "rs_selftest_wait_timeout": [_P, ctypes.c_size_t, _P],
    "rs_trace_read": [ctypes.POINTER(RsTraceEntry), _U32, ctypes.POINTER(ctypes.c_uint32)],
    "rs_set_default_plan": [_U32, _U32, _PLANP],
    "rs_sample_overlap": [_P, _U64, _U32, _U32, _U32, _U32, _U32, _P, ctypes.POINTER(ctypes.c_uint32), _P],
    "rs_choose_plan": [_P, _U64, _PLANP, _PLANP, ctypes.POINTER(ctypes.c_uint32), _P],
    "rs_get_default_plan": [_U32, _U32, _PLANP, ctypes.POINTER(ctypes.c_int)],
}


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIBRARY_PATH):
        raise ImportError(f"{LIBRARY_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    # the CUDA runtime the library links against is the one torch loaded
    import torch  # noqa: F401
    dll = ctypes.CDLL(LIBRARY_PATH)
    for name, args in _SIGS.items():
        f = getattr(dll, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "rs_last_error" else ctypes.c_int
    return dll


lib = _load()


def rs_last_error() -> str:
    return lib.rs_last_error().decode()


def rs_version() -> int:
    return int(lib.rs_version())


def _check(status: int) -> None:
    if status != 0:
        raise RsError(status, rs_last_error())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _plan(plan) -> ctypes.POINTER(RsPlan) | None:
    if plan is None:
        return None
    if isinstance(plan, RsPlan):
        return ctypes.pointer(plan)
    return ctypes.pointer(RsPlan(int(plan.get("digit_bits", 0)), int(plan.get("mode", 0)),
                                 int(plan.get("tile", 0)), int(plan.get("key_kind", 0))))


def _temp(temp):
    if temp is None:
        return None, ctypes.c_size_t(0)
    return _ptr(temp), ctypes.c_size_t(temp.numel() * temp.element_size())


# ------------------------------------------------------------- C entry points
def rs_sort_u32(keys_in, keys_out, n: int, num_parts: int = 64, plan=None, temp=None,
                stream=None, want_offsets: bool = True):
    """Calls rs_sort_u32.  With temp=None it is the size query and returns
    the bytes needed; otherwise it returns the partition offsets (numpy
    uint64[num_parts + 1]) or None."""
    tp, tb = _temp(temp)
    offs = np.zeros(num_parts + 1, dtype=np.uint64) if (want_offsets and temp is not None) else None
    op = offs.ctypes.data_as(_U64P) if offs is not None else None
    _check(lib.rs_sort_u32(_ptr(keys_in), _ptr(keys_out), n, num_parts, op, _plan(plan), tp,
                           ctypes.byref(tb), _stream(stream) if temp is not None else None))
    return tb.value if temp is None else offs


def rs_sort_u32_pairs(keys_in, vals_in, keys_out, vals_out, n: int, num_parts: int = 64, plan=None,
                      temp=None, stream=None, want_offsets: bool = True):
    """Calls rs_sort_u32_pairs; returns as rs_sort_u32."""
    tp, tb = _temp(temp)
    offs = np.zeros(num_parts + 1, dtype=np.uint64) if (want_offsets and temp is not None) else None
    op = offs.ctypes.data_as(_U64P) if offs is not None else None
    _check(lib.rs_sort_u32_pairs(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), n, num_parts,
                                 op, _plan(plan), tp, ctypes.byref(tb),
                                 _stream(stream) if temp is not None else None))
    return tb.value if temp is None else offs


def rs_sort_u64(keys_in, keys_out, n: int, num_parts: int = 64, plan=None, temp=None, stream=None,
                want_offsets: bool = True):
    """Calls rs_sort_u64 (64-bit keys in int64 / uint64 / float64 tensors);
    returns as rs_sort_u32."""
    tp, tb = _temp(temp)
    offs = np.zeros(num_parts + 1, dtype=np.uint64) if (want_offsets and temp is not None) else None
    op = offs.ctypes.data_as(_U64P) if offs is not None else None
    _check(lib.rs_sort_u64(_ptr(keys_in), _ptr(keys_out), n, num_parts, op, _plan(plan), tp, ctypes.byref(tb),
                           _stream(stream) if temp is not None else None))
    return tb.value if temp is None else offs


def rs_sort_u64_pairs(keys_in, vals_in, keys_out, vals_out, n: int, num_parts: int = 64, plan=None, temp=None,
                      stream=None, want_offsets: bool = True):
    """Calls rs_sort_u64_pairs; returns as rs_sort_u32."""
    tp, tb = _temp(temp)
    offs = np.zeros(num_parts + 1, dtype=np.uint64) if (want_offsets and temp is not None) else None
    op = offs.ctypes.data_as(_U64P) if offs is not None else None
    _check(lib.rs_sort_u64_pairs(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), n, num_parts, op,
                                 _plan(plan), tp, ctypes.byref(tb), _stream(stream) if temp is not None else None))
    return tb.value if temp is None else offs


def rs_sort_u64_pairs64(keys_in, vals_in, keys_out, vals_out, n: int, num_parts: int = 64, plan=None, temp=None,
                        stream=None, want_offsets: bool = True):
    """Calls rs_sort_u64_pairs64 (64-bit keys, 64-bit values); returns as
    rs_sort_u32."""
    tp, tb = _temp(temp)
    offs = np.zeros(num_parts + 1, dtype=np.uint64) if (want_offsets and temp is not None) else None
    op = offs.ctypes.data_as(_U64P) if offs is not None else None
    _check(lib.rs_sort_u64_pairs64(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), n, num_parts,
                                   op, _plan(plan), tp, ctypes.byref(tb),
                                   _stream(stream) if temp is not None else None))
    return tb.value if temp is None else offs


def sort64_pairs(keys, vals, num_parts: int = 64, plan=None, stream=None):
    """Stable sort of CUDA tensors of 64-bit keys and 32-bit or (by the
    values' element size) 64-bit values: (keys, vals, host partition
    offsets)."""
    import torch
    n = keys.numel()
    ko, vo = torch.empty_like(keys), torch.empty_like(vals)
    call = rs_sort_u64_pairs64 if vals.element_size() == 8 else rs_sort_u64_pairs
    temp = _alloc_temp(call(None, None, None, None, n, plan=plan), keys.device)
    offs = call(keys, vals, ko, vo, n, num_parts, plan, temp, stream)
    return ko, vo, offs


def rs_sort_u32_pairs64(keys_in, vals_in, keys_out, vals_out, n: int, num_parts: int = 64, plan=None, temp=None,
                        stream=None, want_offsets: bool = True):
    """Calls rs_sort_u32_pairs64 (32-bit keys, 64-bit values); returns as
    rs_sort_u32."""
    tp, tb = _temp(temp)
    offs = np.zeros(num_parts + 1, dtype=np.uint64) if (want_offsets and temp is not None) else None
    op = offs.ctypes.data_as(_U64P) if offs is not None else None
    _check(lib.rs_sort_u32_pairs64(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), n, num_parts,
                                   op, _plan(plan), tp, ctypes.byref(tb),
                                   _stream(stream) if temp is not None else None))
    return tb.value if temp is None else offs


def sort_pairs64(keys, vals, num_parts: int = 64, plan=None, stream=None):
    """Stable (32-bit key, 64-bit value) sort of CUDA tensors: (keys, vals,
    host partition offsets)."""
    import torch
    n = keys.numel()
    ko, vo = torch.empty_like(keys), torch.empty_like(vals)
    temp = _alloc_temp(rs_sort_u32_pairs64(None, None, None, None, n, plan=plan), keys.device)
    offs = rs_sort_u32_pairs64(keys, vals, ko, vo, n, num_parts, plan, temp, stream)
    return ko, vo, offs


def sort64(keys, num_parts: int = 64, plan=None, out=None, temp=None, stream=None):
    """Sorted copy of a CUDA tensor of 64-bit keys (int64 storage of uint64
    keys by default; plan={"key_kind": RS_KEY_I32 or RS_KEY_F32} for signed
    or binary64 keys) and the host partition offsets."""
    import torch
    n = keys.numel()
    out = torch.empty_like(keys) if out is None else out
    if temp is None:
        temp = _alloc_temp(rs_sort_u64(None, None, n, plan=plan), keys.device)
    offs = rs_sort_u64(keys, out, n, num_parts, plan, temp, stream)
    return out, offs


def rs_merge_u32(a, va, na: int, b, vb, nb: int, out, vout, num_parts: int = 64, plan=None, temp=None,
                 stream=None, want_offsets: bool = True):
    """Calls rs_merge_u32; returns as rs_sort_u32."""
    tp, tb = _temp(temp)
    offs = np.zeros(num_parts + 1, dtype=np.uint64) if (want_offsets and temp is not None) else None
    op = offs.ctypes.data_as(_U64P) if offs is not None else None
    _check(lib.rs_merge_u32(_ptr(a), _ptr(va), na, _ptr(b), _ptr(vb), nb, _ptr(out), _ptr(vout), num_parts, op,
                            _plan(plan), tp, ctypes.byref(tb), _stream(stream) if temp is not None else None))
    return tb.value if temp is None else offs


def merge(a, b, va=None, vb=None, num_parts: int = 64, plan=None, stream=None):
    """Stable merge of two sorted CUDA tensors of 32-bit keys (and their
    payloads): (keys, vals or None, host partition offsets)."""
    import torch
    na, nb = a.numel(), b.numel()
    out = torch.empty(na + nb, dtype=a.dtype, device=a.device)
    vout = None if va is None else torch.empty(na + nb, dtype=va.dtype, device=a.device)
    temp = _alloc_temp(rs_merge_u32(None, va, na, None, vb, nb, None, vout, num_parts, plan), a.device)
    offs = rs_merge_u32(a, va, na, b, vb, nb, out, vout, num_parts, plan, temp, stream)
    return out, vout, offs


def rs_sort_u32_host(h_keys_in, h_vals_in, h_keys_out, h_vals_out, n: int, num_parts: int = 64, plan=None,
                     temp=None, stream=None, want_offsets: bool = True):
    """Calls rs_sort_u32_host: the h_* arguments are HOST tensors (CPU,
    preferably pinned) or raw host addresses; temp is a device tensor.
    Returns as rs_sort_u32."""
    tp, tb = _temp(temp)
    offs = np.zeros(num_parts + 1, dtype=np.uint64) if (want_offsets and temp is not None) else None
    op = offs.ctypes.data_as(_U64P) if offs is not None else None
    _check(lib.rs_sort_u32_host(_ptr(h_keys_in), _ptr(h_vals_in), _ptr(h_keys_out), _ptr(h_vals_out), n,
                                num_parts, op, _plan(plan), tp, ctypes.byref(tb),
                                _stream(stream) if temp is not None else None))
    return tb.value if temp is None else offs


def rs_sort_u32_segmented(keys_in, vals_in, keys_out, vals_out, d_seg_offsets, h_seg_offsets,
                          num_segs: int, total_n: int, num_parts: int = 64, d_part_offsets=None,
                          plan=None, temp=None, stream=None):
    """Calls rs_sort_u32_segmented (h_seg_offsets: numpy uint64[num_segs+1]).
    With temp=None returns the bytes needed."""
    tp, tb = _temp(temp)
    h = np.ascontiguousarray(h_seg_offsets, dtype=np.uint64)
    _check(lib.rs_sort_u32_segmented(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out),
                                     _ptr(d_seg_offsets), h.ctypes.data_as(_U64P), num_segs, total_n,
                                     num_parts, _ptr(d_part_offsets), _plan(plan), tp, ctypes.byref(tb),
                                     _stream(stream) if temp is not None else None))
    return tb.value if temp is None else None


def rs_digit_histograms(keys, n: int, digit_bits: int, d_hist, d_bases=None, d_skip=None, stream=None):
    _check(lib.rs_digit_histograms(_ptr(keys), n, digit_bits, _ptr(d_hist), _ptr(d_bases), _ptr(d_skip),
                                   _stream(stream)))


def rs_radix_pass(keys_in, vals_in, keys_out, vals_out, n: int, shift: int, width: int, temp=None,
                  stream=None):
    tp, tb = _temp(temp)
    _check(lib.rs_radix_pass(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), n, shift, width,
                             tp, ctypes.byref(tb), _stream(stream) if temp is not None else None))
    return tb.value if temp is None else None


def rs_sort_u32_noalloc(keys_in, keys_out, n: int, num_parts: int = 64, stream=None,
                        want_offsets: bool = True):
    """Calls rs_sort_u32_noalloc: the keys-only sort with the library's own
    fixed scratch (no device allocation; n <= RS_NOALLOC_MAX_KEYS).  Returns
    the partition offsets (numpy uint64[num_parts + 1]) or None."""
    offs = np.zeros(num_parts + 1, dtype=np.uint64) if want_offsets else None
    op = offs.ctypes.data_as(_U64P) if offs is not None else None
    _check(lib.rs_sort_u32_noalloc(_ptr(keys_in), _ptr(keys_out), n, num_parts, op, _stream(stream)))
    return offs


RS_ENTRY_SORT_U32, RS_ENTRY_SORT_U32_PAIRS, RS_ENTRY_SEGMENTED, RS_ENTRY_SEGMENTED_PAIRS = 0, 1, 2, 3


def rs_sample_overlap(keys, n: int, key_kind: int = 0, bits: int = 13, sample: int = 1000, cells: int = 64,
                      max_problem: int = 2, d_buckets=None, stream=None) -> dict:
    """The selection step of Sec. 4.2.1 on device keys (see include/rsort.h):
    {"problem_cells", "clustered", "shift", "sample"}."""
    out = (ctypes.c_uint32 * 4)()
    _check(lib.rs_sample_overlap(_ptr(keys), n, key_kind, bits, sample, cells, max_problem, _ptr(d_buckets), out,
                                 _stream(stream)))
    return {"problem_cells": int(out[0]), "clustered": bool(out[1]), "shift": int(out[2]), "sample": int(out[3])}


def rs_choose_plan(keys, n: int, plan=None, stream=None) -> tuple[dict, dict]:
    """The plan rs_sort_u32 would run for these keys, chosen by the sample
    of Sec. 4.2.1, and the selection's statistics."""
    out = RsPlan()
    st = (ctypes.c_uint32 * 4)()
    _check(lib.rs_choose_plan(_ptr(keys), n, _plan(plan), ctypes.byref(out), st, _stream(stream)))
    return ({"digit_bits": out.digit_bits, "mode": out.mode, "tile": out.tile, "key_kind": out.key_kind},
            {"problem_cells": int(st[0]), "clustered": bool(st[1]), "shift": int(st[2]), "sample": int(st[3])})


def rs_set_default_plan(entry: int, size_class: int, plan) -> None:
    """Installs (plan dict or RsPlan) or removes (None) the plan an entry
    point uses for a size class when called without one."""
    _check(lib.rs_set_default_plan(entry, size_class, _plan(plan)))


def rs_get_default_plan(entry: int, size_class: int):
    """The installed plan of (entry, size_class) as a dict, or None."""
    out = RsPlan()
    is_set = ctypes.c_int(0)
    _check(lib.rs_get_default_plan(entry, size_class, ctypes.byref(out), ctypes.byref(is_set)))
    if not is_set.value:
        return None
    return {"digit_bits": out.digit_bits, "mode": out.mode, "tile": out.tile}


def rs_check_device_error(stream=None) -> None:
    _check(lib.rs_check_device_error(_stream(stream)))


def rs_peek_device_error_async(h_word, stream=None) -> None:
    """Enqueues a copy of the device error word into h_word (a pinned CPU
    tensor of at least 4 bytes); see include/rsort.h."""
    if h_word.device.type != "cpu" or h_word.numel() * h_word.element_size() < 4:
        raise ValueError("h_word must be a CPU tensor of at least 4 bytes")
    _check(lib.rs_peek_device_error_async(_ptr(h_word), _stream(stream)))


def rs_selftest_wait_timeout(temp, stream=None) -> None:
    """Runs the bounded-wait self-test (see include/rsort.h)."""
    _check(lib.rs_selftest_wait_timeout(_ptr(temp), temp.numel() * temp.element_size(), _stream(stream)))


def rs_trace_enable(on: bool = True) -> None:
    _check(lib.rs_trace_enable(1 if on else 0))


def rs_trace_read() -> dict:
    """{kernel kind: {"launches", "total_ms", "keys"}} since the last read."""
    buf = (RsTraceEntry * 32)()
    cnt = ctypes.c_uint32(0)
    _check(lib.rs_trace_read(buf, 32, ctypes.byref(cnt)))
    return {buf[i].name.decode(): {"launches": int(buf[i].launches), "total_ms": float(buf[i].total_ms),
                                   "keys": float(buf[i].keys)} for i in range(cnt.value)}


# --------------------------------------------------------------- conveniences
def _empty_u32(n, device, like=None):
    """An output buffer of n 32-bit words (the input's dtype when given:
    int32 storage of uint32 keys, or float32 / int32 keys of another kind)."""
    import torch
    dtype = like.dtype if like is not None and like.element_size() == 4 else torch.int32
    return torch.empty(max(n, 0), dtype=dtype, device=device)


def temp_bytes(n: int, pairs: bool = False, plan=None) -> int:
    if pairs:
        return rs_sort_u32_pairs(None, None, None, None, n, plan=plan)
    return rs_sort_u32(None, None, n, plan=plan)


def _alloc_temp(nbytes: int, device):
    import torch
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)


def sort(keys, num_parts: int = 64, plan=None, out=None, temp=None, stream=None):
    """Sorted copy of a CUDA tensor of 32-bit keys (uint32 in int32 storage by
    default; plan={"key_kind": RS_KEY_I32 or RS_KEY_F32} for signed or float
    keys) and the host partition offsets."""
    n = keys.numel()
    out = _empty_u32(n, keys.device, keys) if out is None else out
    if temp is None:
        temp = _alloc_temp(rs_sort_u32(None, None, n, plan=plan), keys.device)
    offs = rs_sort_u32(keys, out, n, num_parts, plan, temp, stream)
    return out, offs


def sort_pairs(keys, vals, num_parts: int = 64, plan=None, out_keys=None, out_vals=None, temp=None,
               stream=None):
    n = keys.numel()
    ko = _empty_u32(n, keys.device, keys) if out_keys is None else out_keys
    vo = _empty_u32(n, keys.device, vals) if out_vals is None else out_vals
    if temp is None:
        temp = _alloc_temp(rs_sort_u32_pairs(None, None, None, None, n, plan=plan), keys.device)
    offs = rs_sort_u32_pairs(keys, vals, ko, vo, n, num_parts, plan, temp, stream)
    return ko, vo, offs


def sort_segmented(keys, vals, seg_offsets_host, num_parts: int = 64, plan=None, temp=None, stream=None,
                   want_part_offsets: bool = True):
    """Segmented sort; seg_offsets_host is a numpy uint64 array (num_segs+1)."""
    import torch
    h = np.ascontiguousarray(seg_offsets_host, dtype=np.uint64)
    num_segs = h.size - 1
    total = int(h[-1]) if h.size else 0
    dev = keys.device
    d_seg = torch.from_numpy(h.view(np.int64)).to(dev)
    ko = _empty_u32(total, dev, keys)
    vo = _empty_u32(total, dev, vals) if vals is not None else None
    po = torch.empty(num_segs * (num_parts + 1), dtype=torch.int64, device=dev) if want_part_offsets else None
    if temp is None:
        nb = rs_sort_u32_segmented(None, vals, None, vo, None, h, num_segs, total, num_parts, plan=plan)
        temp = _alloc_temp(nb, dev)
    rs_sort_u32_segmented(keys, vals, ko, vo, d_seg, h, num_segs, total, num_parts, po, plan, temp, stream)
    return ko, vo, po
