"""The stronger CPU baseline (not the oracle): an LSD radix sort of uint32
keys on all host threads, in C (``cpu_radix.c``).  Test infrastructure like
the rest of this package: ``bench.py`` times it beside the single-thread
oracle, and ``tests/`` check it against the oracle.

``build_library()`` compiles ``cpu_radix.c`` in place (gcc, -O3, POSIX
threads); ``sort(keys, threads)`` sorts a numpy uint32 array with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(HERE, "cpu_radix.c")
LIBRARY = os.path.join(HERE, "libcpuradix.so")
_lib = None


def build_library() -> str:
    """Compiles cpu_radix.c into libcpuradix.so next to it when the library
    is missing or older than the source.  Returns the library's path."""
    if not os.path.exists(LIBRARY) or os.path.getmtime(LIBRARY) < os.path.getmtime(SOURCE):
        tmp = LIBRARY + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-pthread", SOURCE, "-o", tmp], check=True)
        os.replace(tmp, LIBRARY)
    return LIBRARY


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_library())
        lib.cpu_radix_sort_u32.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                           ctypes.c_int]
        lib.cpu_radix_sort_u32.restype = ctypes.c_int
        _lib = lib
    return _lib


def default_threads() -> int:
    return max(1, min(256, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()))


def sort(keys: np.ndarray, threads: int | None = None, out: np.ndarray | None = None,
         tmp: np.ndarray | None = None) -> np.ndarray:
    """The keys (uint32) in ascending order, sorted on `threads` host threads
    (default: every core this process may run on).  `out` / `tmp` may be
    given (n uint32 each) to keep allocation out of a timed loop."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    n = keys.size
    out = np.empty(n, np.uint32) if out is None else out
    tmp = np.empty(n, np.uint32) if tmp is None else tmp
    t = default_threads() if threads is None else int(threads)
    rc = _load().cpu_radix_sort_u32(keys.ctypes.data, out.ctypes.data, tmp.ctypes.data, n, t)
    if rc != 0:
        raise RuntimeError("cpu_radix_sort_u32 failed")
    return out
