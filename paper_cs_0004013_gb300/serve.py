"""A sort-serving loop with continuous batching.

Requests (uint32 keys, optionally uint32 payloads) arrive over time.  At
each scheduler tick, the requests that have arrived are admitted while a slot
is free and the device-memory budget allows; each admitted group becomes one
batch: its requests are copied (pinned host -> device) into one arena, sorted
by a single ``rs_sort_u32_segmented`` call (each request is one segment), and
copied back (device -> pinned host), all on one of ``streams`` CUDA streams
(one that no batch in flight uses), so batches formed at different ticks
overlap on the device.  A request of at
least ``direct_min_keys`` keys forms a batch of its own, sorted by one
``rs_sort_u32_host`` call straight from and into its pinned buffers (the
plain sort's kernels, no arena); one such batch's copy back then overlaps the
next one's copy in and sort.  A request's
latency is the time from its arrival to the moment its result is back on the
host (the batch's completion event).  Buffers stay resident: arenas and temp
are reused from a pool keyed by size class.

PyTorch is used for device memory, pinned host memory, streams and events
only; all sorting runs in librsort's kernels.  Each request's result does not
depend on what it was batched with (the segmented sort treats every segment
on its own), which ``tests/test_gpu_serve.py`` checks bit for bit.

After each batch's work its stream copies the device error word (bounded
waits that gave up, output-index checks that fired) into a pinned word,
asynchronously; when the batch completes, the server reads that copy, and
only if a bit is set does it take and clear the word (on a stream of its
own).  The word is shared by every stream of the device, so an error cannot
be pinned on one batch: the completed batch and every batch still in flight
at that moment are marked failed (``Request.error``), and ``run`` returns
with ``failed`` counting them instead of reporting wrong results as served.
"""
from __future__ import annotations

import dataclasses
import math
import time
from collections import deque

import numpy as np

from . import (RsError, rs_check_device_error, rs_peek_device_error_async, rs_sort_u32, rs_sort_u32_host,
               rs_sort_u32_pairs, rs_sort_u32_segmented)

__all__ = ["Request", "ResultPool", "SortServer", "serial_plain", "latency_stats"]


@dataclasses.dataclass
class Request:
    """One sort request.  keys / vals are pinned host tensors (int32 storage
    of uint32 values) owned by the client; the server copies them to the
    device and the sorted result back into out_keys / out_vals (pinned,
    allocated with the request, or lent by the server's ResultPool until
    on_done returns), with no host-side copy in between."""
    id: int
    arrival_s: float           # offset from the start of the run
    keys: object               # pinned torch.int32 [n]
    vals: object = None        # pinned torch.int32 [n] or None
    out_keys: object = None
    out_vals: object = None
    done_s: float | None = None
    batch: int | None = None
    error: str | None = None   # set when the device reported an error for the request's batch
    pooled: object = dataclasses.field(default=None, repr=False)  # result buffers lent by a ResultPool

    @staticmethod
    def make(rid: int, arrival_s: float, keys: np.ndarray, vals: np.ndarray | None = None) -> "Request":
        import torch
        k = torch.from_numpy(np.ascontiguousarray(keys).view(np.int32)).pin_memory()
        v = None if vals is None else torch.from_numpy(np.ascontiguousarray(vals).view(np.int32)).pin_memory()
        r = Request(rid, arrival_s, k, v)
        r.out_keys = torch.empty_like(k).pin_memory()
        r.out_vals = None if v is None else torch.empty_like(v).pin_memory()
        return r

    @staticmethod
    def view(rid: int, arrival_s: float, keys, vals=None) -> "Request":
        """A request over pinned int32 tensors the client already holds (for
        example slices of one pinned pool).  Its result buffers are left
        unset: a server with a result pool hands them out at admission."""
        return Request(rid, arrival_s, keys, vals)

    @property
    def n(self) -> int:
        return int(self.keys.numel())

    @property
    def pairs(self) -> bool:
        return self.vals is not None

    def bytes_needed(self) -> int:
        return self.n * 4 * (4 if self.pairs else 2)

    def result(self):
        """(keys, vals or None) as numpy uint32 arrays."""
        k = self.out_keys.numpy().view(np.uint32)
        return k, (None if self.out_vals is None else self.out_vals.numpy().view(np.uint32))


def _size_class(nbytes: int) -> int:
    return 1 << max(20, math.ceil(math.log2(max(nbytes, 1))))


class _Pool:
    """Device buffers reused by size class (powers of two, >= 1 MiB)."""

    def __init__(self, device):
        self.device = device
        self.free: dict[int, list] = {}
        self.bytes_held = 0

    def take(self, nbytes: int):
        import torch
        c = _size_class(nbytes)
        lst = self.free.get(c)
        if lst:
            return lst.pop()
        self.bytes_held += c
        return torch.empty(c, dtype=torch.uint8, device=self.device)

    def give(self, buf):
        self.free.setdefault(buf.numel(), []).append(buf)


class ResultPool:
    """Pinned host buffers for results, reused by size class, with a cap on
    the bytes handed out at once.  A server given one assigns result buffers
    to requests that have none when it admits them (admission waits while
    the cap is reached), calls the client's on_done(request) when a request
    completes, and then takes its buffers back: the client reads or copies
    the result inside on_done."""

    def __init__(self, max_bytes: int):
        self.max_bytes = max_bytes
        self.out = 0
        self.free: dict[int, list] = {}

    def take(self, nbytes: int):
        import torch
        c = _size_class(nbytes)
        if self.out + c > self.max_bytes and self.out > 0:
            return None
        self.out += c
        lst = self.free.get(c)
        return lst.pop() if lst else torch.empty(c, dtype=torch.uint8).pin_memory()

    def give(self, buf):
        self.out -= buf.numel()
        self.free.setdefault(buf.numel(), []).append(buf)


class _Batch:
    def __init__(self, bid, reqs, pairs, stream, arena, temp, h_in, h_out, done_event, start_event):
        self.id, self.reqs, self.pairs, self.stream = bid, reqs, pairs, stream
        self.arena, self.temp, self.h_in, self.h_out = arena, temp, h_in, h_out
        self.done_event, self.start_event = done_event, start_event
        self.err_word = None  # pinned copy of the device error word, taken after the batch's work


# error-word bits (include/rsort.h, rs_peek_device_error_async)
_ERR_TIMEOUT, _ERR_BOUNDS = 1, 2


class SortServer:
    """Continuous-batching sort server on one GPU.

    slots: batches in flight at most; streams: CUDA streams used round
    robin; mem_budget: bytes of device memory the server may hold for
    in-flight batches (inputs, outputs and temp); max_batch_keys: largest
    batch arena in keys; direct_min_keys: requests this large are sorted on
    their own, from and into their pinned buffers; tuner: a tune.Tuner whose
    cached plans are installed in the library for the server's calls."""

    def __init__(self, slots: int = 8, streams: int = 8, mem_budget: int = 8 << 30,
                 max_batch_keys: int = 1 << 24, num_parts: int = 64, device: str = "cuda",
                 direct_min_keys: int = 1 << 22, result_pool: ResultPool | None = None, on_done=None,
                 tuner=None):
        import torch
        self.result_pool, self.on_done = result_pool, on_done
        # A tuner's cached choices (digit width, tile shape, MSD or LSD per
        # size class) become the library's plans for calls without one: the
        # server's segmented batches and direct sorts pass no plan.
        self.tuned_plans = tuner.install() if tuner is not None else 0
        self.device = torch.device(device)
        self.slots, self.mem_budget, self.max_batch_keys = slots, mem_budget, max_batch_keys
        self.direct_min_keys = direct_min_keys
        self.num_parts = num_parts
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        # the error word is taken on a stream of its own (see _check_errors)
        self.err_stream = torch.cuda.Stream(device=self.device)
        self.err_words: list = []  # pinned 4-byte words for the per-batch peeks
        self.pool = _Pool(self.device)
        self.pinned = {}
        self.in_flight: list[_Batch] = []
        self.mem_in_use = 0
        self.next_batch = 0
        self.t0_event = None
        self.t0_host = None
        self.suspect: dict[int, str] = {}  # batch id -> error seen while it was in flight
        self.failed = 0

    # -- pinned staging buffers, reused by size class
    def _pinned(self, key, nbytes):
        import torch
        c = _size_class(nbytes)
        lst = self.pinned.setdefault((key, c), [])
        if lst:
            return lst.pop()
        return torch.empty(c, dtype=torch.uint8).pin_memory()

    def _return_pinned(self, key, buf):
        self.pinned.setdefault((key, buf.numel()), []).append(buf)

    def _batch_bytes(self, reqs, pairs):
        n = sum(r.n for r in reqs)
        offs = np.zeros(len(reqs) + 1, dtype=np.uint64)
        offs[1:] = np.cumsum([r.n for r in reqs])
        temp = rs_sort_u32_segmented(None, 1 if pairs else None, None, 1 if pairs else None, None, offs,
                                     len(reqs), n, self.num_parts)
        return n * 4 * (4 if pairs else 2) + len(reqs) * 8 + temp, offs, temp

    def _finish_launch(self, b):
        """After a batch's work on its stream: an asynchronous copy of the
        device error word (no kernel, no wait), then the completion event."""
        import torch
        b.err_word = self.err_words.pop() if self.err_words else torch.zeros(1, dtype=torch.int32).pin_memory()
        rs_peek_device_error_async(b.err_word, b.stream)
        b.done_event.record(b.stream)

    def _stream(self):
        """A stream no batch in flight uses (a batch queued behind another on
        its stream would wait for it though the device has room), else the
        next one round robin."""
        busy = {id(b.stream) for b in self.in_flight}
        for k in range(len(self.streams)):
            st = self.streams[(self.next_batch + k) % len(self.streams)]
            if id(st) not in busy:
                return st
        return self.streams[self.next_batch % len(self.streams)]

    def _launch_direct(self, r):
        import torch
        stream = self._stream()
        need = rs_sort_u32_host(None, r.vals, None, r.out_vals, r.n, self.num_parts)
        temp = self.pool.take(need)
        done = torch.cuda.Event()
        rs_sort_u32_host(r.keys, r.vals, r.out_keys, r.out_vals, r.n, self.num_parts, None, temp, stream,
                         want_offsets=False)
        b = _Batch(self.next_batch, [r], r.pairs, stream, None, temp, None, None, done, None)
        self._finish_launch(b)
        r.batch = b.id
        self.next_batch += 1
        self.mem_in_use += need
        b.need = need
        self.in_flight.append(b)

    def _launch(self, reqs, pairs):
        import torch
        if len(reqs) == 1 and reqs[0].n >= self.direct_min_keys:
            return self._launch_direct(reqs[0])
        need, offs, temp_bytes = self._batch_bytes(reqs, pairs)
        n = int(offs[-1])
        stream = self._stream()
        words = n * (2 if pairs else 1)
        arena = self.pool.take(2 * words * 4 + (len(reqs) + 1) * 8)
        temp = self.pool.take(max(temp_bytes, 1))
        h_off = self._pinned("off", (len(reqs) + 1) * 8)
        h_off[: (len(reqs) + 1) * 8].view(torch.int64).numpy()[:] = offs.view(np.int64)
        done = torch.cuda.Event()
        with torch.cuda.stream(stream):
            d_in = arena[: words * 4].view(torch.int32)
            d_out = arena[words * 4: 2 * words * 4].view(torch.int32)
            d_off = arena[2 * words * 4: 2 * words * 4 + (len(reqs) + 1) * 8].view(torch.int64)
            d_off.copy_(h_off[: (len(reqs) + 1) * 8].view(torch.int64), non_blocking=True)
            for i, r in enumerate(reqs):
                a, e = int(offs[i]), int(offs[i + 1])
                d_in[a:e].copy_(r.keys, non_blocking=True)
                if pairs:
                    d_in[n + a: n + e].copy_(r.vals, non_blocking=True)
            kin, kout = d_in[:n], d_out[:n]
            vin = d_in[n:] if pairs else None
            vout = d_out[n:] if pairs else None
            rs_sort_u32_segmented(kin, vin, kout, vout, d_off, offs, len(reqs), n, self.num_parts, None,
                                  None, temp, stream)
            for i, r in enumerate(reqs):
                a, e = int(offs[i]), int(offs[i + 1])
                r.out_keys.copy_(d_out[a:e], non_blocking=True)
                if pairs:
                    r.out_vals.copy_(d_out[n + a: n + e], non_blocking=True)
        b = _Batch(self.next_batch, reqs, pairs, stream, arena, temp, h_off, None, done, None)
        self._finish_launch(b)
        for r in reqs:
            r.batch = b.id
        self.next_batch += 1
        self.mem_in_use += need
        b.need = need
        b.offs = offs
        self.in_flight.append(b)

    def _check_errors(self, b):
        """Batch b's peek of the error word (copied after its work) is read;
        if a bit was set, the word is taken and cleared, and b and every
        batch still in flight (any of them may have raised it) are marked.
        The take runs on the server's own error stream, which holds no
        batch, so it does not wait for the batches queued after b on b's
        stream; when the word is clear (the usual case) nothing waits."""
        word = int(b.err_word[0]) & 0xFFFFFFFF
        self.err_words.append(b.err_word)
        b.err_word = None
        if word == 0:
            return
        what = "RS_ERR_TIMEOUT" if word & _ERR_TIMEOUT else "RS_ERR_CUDA"
        msg = f"{what}: device error word 0x{word:x} after the batch"
        try:
            rs_check_device_error(self.err_stream)
        except RsError as e:
            msg = str(e)
        self.suspect[b.id] = msg
        for o in self.in_flight:
            self.suspect.setdefault(o.id, msg)

    def _assign_results(self, r) -> bool:
        """Gives r result buffers from the pool if it has none; False if the
        pool is at its cap (r waits)."""
        if r.out_keys is not None or self.result_pool is None:
            return True
        kb = self.result_pool.take(r.n * 4)
        if kb is None:
            return False
        vb = None
        if r.pairs:
            vb = self.result_pool.take(r.n * 4)
            if vb is None:
                self.result_pool.give(kb)
                return False
        import torch
        r.pooled = (kb, vb)
        r.out_keys = kb[: r.n * 4].view(torch.int32)
        r.out_vals = None if vb is None else vb[: r.n * 4].view(torch.int32)
        return True

    def _retire(self, b, now_s):
        self._check_errors(b)
        err = self.suspect.pop(b.id, None)
        for r in b.reqs:
            r.done_s = now_s
            r.error = err
            if err is not None:
                self.failed += 1
            if self.on_done is not None:
                self.on_done(r)
            if r.pooled is not None:
                for buf in r.pooled:
                    if buf is not None:
                        self.result_pool.give(buf)
                r.pooled = None
                r.out_keys = r.out_vals = None
        if b.arena is not None:
            self.pool.give(b.arena)
            self._return_pinned("off", b.h_in)
        self.pool.give(b.temp)
        self.mem_in_use -= b.need

    def _poll(self):
        now = time.perf_counter() - self.t0_host
        still = []
        for b in self.in_flight:
            if b.done_event.query():
                self._retire(b, now)
            else:
                still.append(b)
        self.in_flight = still

    def run(self, requests: list[Request], realtime: bool = True) -> list[Request]:
        """Serves `requests` (sorted by arrival).  With realtime=False every
        request counts as arrived at the start (closed-loop throughput)."""
        import torch
        if not realtime:  # closed loop: every request is submitted at the start
            for r in requests:
                r.arrival_s = 0.0
        pending = deque(sorted(requests, key=lambda r: r.arrival_s))
        torch.cuda.synchronize(self.device)
        self.t0_host = time.perf_counter()
        while pending or self.in_flight:
            self._poll()
            now = time.perf_counter() - self.t0_host
            # gather arrived requests into at most two batches (keys / pairs)
            while pending and len(self.in_flight) < self.slots:
                if realtime and pending[0].arrival_s > now:
                    break
                group = {False: [], True: []}
                budget = self.mem_budget - self.mem_in_use
                keys_in_batch = {False: 0, True: 0}
                while pending and (not realtime or pending[0].arrival_s <= now):
                    r = pending[0]
                    if keys_in_batch[r.pairs] + r.n > self.max_batch_keys and group[r.pairs]:
                        break
                    if r.n >= self.direct_min_keys and (group[False] or group[True]):
                        break  # sorted on its own, at the next admission
                    cost = 3 * r.bytes_needed()
                    if cost > budget and (group[False] or group[True] or self.in_flight):
                        break
                    if not self._assign_results(r):
                        break  # the result pool is at its cap: wait for completions
                    group[r.pairs].append(pending.popleft())
                    keys_in_batch[r.pairs] += r.n
                    budget -= cost
                    if r.n >= self.direct_min_keys:
                        break
                if not group[False] and not group[True]:
                    break
                for pairs in (False, True):
                    if group[pairs]:
                        self._launch(group[pairs], pairs)
            if not self.in_flight and pending and realtime:
                wait = pending[0].arrival_s - (time.perf_counter() - self.t0_host)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
            elif self.in_flight:
                time.sleep(0.0001)
        for s in self.streams:
            s.synchronize()
        return requests


def serial_plain(requests: list[Request], num_parts: int = 64, device: str = "cuda") -> float:
    """One request at a time on one stream: its pinned keys (and values) to
    the device, one plain rs_sort_u32(_pairs) call, the result back into its
    pinned output, then wait.  Returns the elapsed seconds."""
    import torch
    dev = torch.device(device)
    big = max(r.n for r in requests)
    d_k = torch.empty(big, dtype=torch.int32, device=dev)
    d_v = torch.empty(big, dtype=torch.int32, device=dev)
    o_k = torch.empty_like(d_k)
    o_v = torch.empty_like(d_k)
    temp = torch.empty(max(rs_sort_u32_pairs(None, None, None, None, big), rs_sort_u32(None, None, big)),
                       dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    # requests without result buffers of their own share one pinned scratch pair
    need_scratch = any(r.out_keys is None for r in requests)
    sk = torch.empty(big, dtype=torch.int32).pin_memory() if need_scratch else None
    sv = torch.empty(big, dtype=torch.int32).pin_memory() if need_scratch else None
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for r in requests:
        n = r.n
        ok_ = r.out_keys if r.out_keys is not None else sk[:n]
        d_k[:n].copy_(r.keys, non_blocking=True)
        if r.pairs:
            d_v[:n].copy_(r.vals, non_blocking=True)
            rs_sort_u32_pairs(d_k, d_v, o_k, o_v, n, num_parts, None, temp, stream)
            (r.out_vals if r.out_vals is not None else sv[:n]).copy_(o_v[:n], non_blocking=True)
        else:
            rs_sort_u32(d_k, o_k, n, num_parts, None, temp, stream)
        ok_.copy_(o_k[:n], non_blocking=True)
        stream.synchronize()
    return time.perf_counter() - t0


def latency_stats(requests: list[Request]) -> dict:
    """p50 / p99 / mean latency of the requests served without a device error."""
    lat = np.array([r.done_s - r.arrival_s for r in requests if r.error is None])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
