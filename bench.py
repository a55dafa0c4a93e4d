"""Throughput of the GB300 radix sort: Gkeys/s sorting 2^26 uint32 keys.

One step = one whole sort (upfront histogram, digit scans, every onesweep
pass) of 2^26 uniform 31-bit keys already resident in HBM, keys only, with
the 64 partition offsets.  The keys (268 MB) exceed the 126 MB L2, so no
flush is needed between steps.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The "e2e" figure sorts host arrays through rs_sort_u32_host: pinned keys
in, sorted keys out, every copy inside the timed region, consecutive sorts
spread over three streams so that their copies overlap.

Beside the headline (default run only) the line carries three more
measured figures: "pairs" (the same keys with a uint32 payload), "batched"
(config 4: ~1.8K uneven key+payload arrays, 2^28 keys, one segmented call
against one plain call per array) and "served" (config 5: 1000 Poisson
requests per offered load, p50/p99 latency, closed-loop keys/s against
serial plain launches).  --no-extra skips them.

--impl reference times the oracle (a plain numpy sort, one host core) on the
same 2^26-key workload (about 5 s per step).  Under torchrun every rank sorts its
own 2^26 keys (replicas: the sort does not shard across GPUs here); the
value is all ranks' keys over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gkeys/s sorting 2^26 u32 on 1 GB300, % HBM roofline; batched/served vs plain"
N_KEYS = 1 << 26
WORKLOAD = "plain sort of 2^26 uint32 keys uniform in [0, 2^31-1], keys only, 64 partitions"


KEY_KINDS = {"u32": 0, "i32": 1, "f32": 2}


def size_text(n: int) -> str:
    """n as a power of two when it is one."""
    return f"2^{n.bit_length() - 1}" if n > 0 and n & (n - 1) == 0 else str(n)


def workload_label(n: int, pairs: bool, key_kind: str = "u32") -> str:
    size = size_text(n)
    w = WORKLOAD.replace("2^26", size)
    if key_kind == "i32":
        w = w.replace("uint32 keys uniform in [0, 2^31-1]", "int32 keys uniform over all 2^32 values")
    elif key_kind == "f32":
        w = w.replace("uint32 keys uniform in [0, 2^31-1]",
                      "float32 keys (uniform 32-bit patterns, IEEE totalOrder)")
    return w.replace("keys only", "key+payload") if pairs else w
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 126 * 1024 * 1024
FLUSH_BYTES = 256 << 20
E2E_STREAMS = 3
CLOCK_SETTLE_S = 1.0
REFERENCE_BUDGET_S = 100.0  # the reference arm's whole run


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_KEYS, help="keys per sort (default 2^26)")
    ap.add_argument("--digit-bits", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--mode", choices=["auto", "lsd", "msd"], default="auto",
                    help="msd: bucket by bits 18-31, then sort each bucket (the MSD plan)")
    ap.add_argument("--pairs", action="store_true", help="time key+payload sorts as the main value")
    ap.add_argument("--keys64", action="store_true", help="64-bit keys (rs_sort_u64), uniform over all 2^64 words")
    ap.add_argument("--vals64", action="store_true",
                    help="32-bit keys with 64-bit values (rs_sort_u32_pairs64) as the main value")
    ap.add_argument("--key-kind", choices=["u32", "i32", "f32"], default="u32",
                    help="how the 32-bit key words are ordered (u32: the headline workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["plain", "batched", "serve", "dist", "merge"], default="plain",
                    help="plain: the headline 2^26 sort; batched: 4096 log-uniform segments in one call vs one "
                         "call per array; serve: Poisson request stream; dist: the four skewed 2^26 inputs")
    ap.add_argument("--requests", type=int, default=1000, help="requests per load point (serve)")
    ap.add_argument("--no-extra", action="store_true",
                    help="plain workload: skip the key+payload, batched and served figures beside the main value")
    return ap.parse_args()


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 100 ms, each stamped with the host time it
    arrived, so that the samples of a time window can be picked out."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.samples = []  # (time.monotonic() on arrival, csv line)
        self._reader = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        if self.proc is not None:
            self._reader = threading.Thread(target=self._read, daemon=True)
            self._reader.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self.samples.append((time.monotonic(), line))

    def wait_first(self, timeout_s: float = 3.0):
        """Returns once the first sample has arrived (or after timeout_s)."""
        end = time.monotonic() + timeout_s
        while self.proc is not None and not self.samples and time.monotonic() < end:
            time.sleep(0.01)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self._reader is not None:
                self._reader.join(timeout=5)

    def summary(self, window=None, timed=None):
        """Median SM clock and the throttle reasons seen over the samples that
        arrived inside `window` (all samples if None); `timed` counts the
        samples inside the timed region itself."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        picked = [l for t, l in self.samples if window is None or window[0] <= t <= window[1]]
        for l in picked:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": sorted(reasons), "samples": len(sm)}
        if timed is not None:
            out["samples_in_timed_region"] = sum(1 for t, _ in self.samples if timed[0] <= t <= timed[1])
        return out


# ------------------------------------------------------------ cpu baseline
def workload_keys(n: int, seed: int, key_kind: str) -> np.ndarray:
    """The timed workload's keys: uniform 31-bit keys (the headline), or
    for signed / binary32 kinds every 32-bit pattern (both signs; NaNs,
    infinities and denormals for binary32)."""
    import synth
    if key_kind == "u32":
        return synth.uniform31(n, seed)
    if key_kind == "u64":
        return synth.splitmix64(seed, n)
    return synth.splitmix64(seed, (n + 1) // 2).view(np.uint32)[:n].copy()


def sorted_by_kind(keys: np.ndarray, key_kind: str) -> np.ndarray:
    """Sanity reference for the end-to-end check (not the oracle): the words
    in order of their kind through the order-preserving unsigned map."""
    f, m = {"u32": (0, 0), "i32": (0, 0x80000000), "f32": (0x7FFFFFFF, 0x80000000)}[key_kind]
    sign = (keys >> np.uint32(31)).astype(bool)
    t = np.sort(keys ^ (np.where(sign, np.uint32(f), np.uint32(0)) ^ np.uint32(m)))
    top = (t >> np.uint32(31)).astype(bool)  # the complement of the original sign
    return t ^ (np.where(top, np.uint32(0), np.uint32(f)) ^ np.uint32(m))


def cpu_parallel_baseline(sample_keys: int = N_KEYS, reps: int = 5):
    """The stronger CPU baseline (not the oracle): an LSD radix sort of the
    workload's 2^26 keys on every host core (C, POSIX threads; oracle/
    cpu_radix.c), timed over `reps` whole sorts after one untimed sort."""
    import synth
    from oracle import cpu_baseline as cb
    keys = workload_keys(sample_keys, synth.CONFIG_SEED + 2, "u32")
    out, tmp = np.empty_like(keys), np.empty_like(keys)
    threads = cb.default_threads()
    cb.sort(keys, threads, out, tmp)
    t0 = time.perf_counter()
    for _ in range(reps):
        cb.sort(keys, threads, out, tmp)
    el = time.perf_counter() - t0
    if not np.array_equal(out[:: max(1, sample_keys // 4096)], np.sort(keys)[:: max(1, sample_keys // 4096)]):
        raise SystemExit("the CPU radix baseline did not sort")
    return {"value": reps * sample_keys / el / 1e9, "unit": "Gkeys/s", "cores": threads,
            "host_cores": os.cpu_count(), "kind": "parallel LSD radix sort, 8-bit digits (C, POSIX threads)",
            "sample": f"{reps} whole sorts of the workload's 2^26 keys, {el:.2f} s"}


def cpu_baseline(sample_keys: int = N_KEYS, budget_s: float = 12.0, key_kind: str = "u32"):
    """The oracle as it stands (numpy stable sort, one core) on the
    workload itself: whole sorts of its 2^26 keys, at least two, until the
    time budget is spent.  `cores` is what the oracle uses (one thread);
    `host_cores` what the host offers."""
    import oracle
    import synth
    keys = workload_keys(sample_keys, synth.CONFIG_SEED + 2, key_kind)
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.sort_keys(keys, key_kind)
        reps += 1
        el = time.perf_counter() - t0
        if (el > budget_s and reps >= 2) or reps >= 50:
            break
    rate = reps * sample_keys / el / 1e9
    size = f"2^{sample_keys.bit_length() - 1}" if sample_keys & (sample_keys - 1) == 0 else str(sample_keys)
    return {"value": rate, "unit": "Gkeys/s", "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{reps} whole sorts of the workload's {size} keys ({key_kind}; numpy stable sort, "
                      f"one thread), {el:.1f} s"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synth
    total = args.n  # the workload's keys (2^26 by default)
    keys = synth.uniform31(total, synth.CONFIG_SEED + 2)  # the workload itself
    # Each step sorts a prefix of the workload's keys, as long as the whole
    # run fits REFERENCE_BUDGET_S (the oracle takes seconds per 2^26 keys):
    # the prefix is the longest power of two whose estimated time, scaled
    # from one timed sort of up to 2^20 keys, fits the steps plus one warm-up.
    probe = min(total, 1 << 20)
    t0 = time.perf_counter()
    oracle.sort_keys(keys[:probe])
    per_key = (time.perf_counter() - t0) / max(probe, 1) * 1.3  # n log n growth up to 2^26
    size = total
    while size > (1 << 20) and (args.steps + min(args.warmup, 1)) * size * per_key > REFERENCE_BUDGET_S:
        size //= 2
    sample = keys[:size]
    for _ in range(min(args.warmup, 1)):
        oracle.sort_keys(sample)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sort_keys(sample)
        t.append(time.perf_counter() - t0)
    tot = sum(t)
    rate = args.steps * sample.size / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "Gkeys/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": workload_label(total, False), "keys_per_step": int(sample.size)},
            "cpu_baseline": {"value": rate, "unit": "Gkeys/s", "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"each step sorts the first {size_text(sample.size)} of the workload's "
                                       f"{size_text(total)} uniform 31-bit keys (numpy stable sort, one host "
                                       "thread); at most one warm-up sort"},
            "e2e": {"value": rate, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- replicas
def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (the job's time) when ranks run replicas."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(keys_per_rank: int, world: int, steps: int, job_ms: float) -> float:
    """Gkeys/s of the whole job: every rank's keys over the slowest time."""
    return world * keys_per_rank * steps / (job_ms * 1e-3) / 1e9


# ------------------------------------------------------------------ ours
PASS_SOURCES = ("onesweep.cuh", "onesweep2.cuh", "onesweep_r8.cu")


def pass_kernel_sha() -> str:
    """First 16 hex digits of the sha256 of the 8-bit pass kernels' sources
    (both kernel forms and the tile-shape registry that picks between them)."""
    h = hashlib.sha256()
    for f in PASS_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_cs_0004013_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profiles(key: str):
    """DRAM bytes per launch recorded by ncu for the pass kernel, valid only
    while the pass kernels' sources are unchanged (their sha256 is stored
    with the figure)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        sha = pass_kernel_sha()
        for line in open(path):
            f = line.split()
            if len(f) >= 3 and f[0] == key and f[1] == sha:
                return float(f[2])
    except OSError:
        pass
    return None


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    # The served form runs first, in a process of its own, before this one
    # touches the GPU (see measure_served_in_own_process).
    served = None
    if (world == 1 and not args.no_extra and not args.keys64 and not args.vals64 and not args.pairs
            and args.key_kind == "u32" and args.n == N_KEYS and not args.digit_bits and not args.tile
            and args.mode == "auto"):
        served = measure_served_in_own_process(args.requests)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import synth
    import paper_cs_0004013_gb300 as rs

    dev = torch.device("cuda", torch.cuda.current_device())
    n = args.n
    wide = args.keys64
    if wide:  # uniform 64-bit words
        keys = workload_keys(n, synth.CONFIG_SEED + 2 + 1000 * rank, "u64")
        d_keys = torch.from_numpy(keys.view(np.int64)).to(dev)
    else:
        keys = workload_keys(n, synth.CONFIG_SEED + 2 + 1000 * rank, args.key_kind)
        d_keys = torch.from_numpy(keys.view(np.int32)).to(dev)
    d_out = torch.empty_like(d_keys)
    plan = {"digit_bits": args.digit_bits, "tile": args.tile, "key_kind": KEY_KINDS[args.key_kind],
            "mode": {"auto": 0, "lsd": 1, "msd": 2}[args.mode]}
    vals64 = args.vals64 and not wide
    wide_v64 = args.vals64 and wide  # 64-bit keys with 64-bit values
    pairs = args.pairs or args.vals64
    if wide_v64:
        d_vals = torch.arange(n, dtype=torch.int64, device=dev)
        d_vout = torch.empty_like(d_vals)
        temp = torch.empty(rs.rs_sort_u64_pairs64(None, None, None, None, n, plan=plan), dtype=torch.uint8,
                           device=dev)
    elif vals64:
        d_vals = torch.arange(n, dtype=torch.int64, device=dev)
        d_vout = torch.empty_like(d_vals)
        temp = torch.empty(rs.rs_sort_u32_pairs64(None, None, None, None, n, plan=plan), dtype=torch.uint8,
                           device=dev)
    elif wide:
        if pairs:
            d_vals = torch.arange(n, dtype=torch.int32, device=dev)
            d_vout = torch.empty_like(d_vals)
            nb = rs.rs_sort_u64_pairs(None, None, None, None, n, plan=plan)
        else:
            nb = rs.rs_sort_u64(None, None, n, plan=plan)
        temp = torch.empty(nb, dtype=torch.uint8, device=dev)
    elif pairs:
        d_vals = torch.arange(n, dtype=torch.int32, device=dev)
        d_vout = torch.empty_like(d_vals)
        temp = torch.empty(rs.rs_sort_u32_pairs(None, None, None, None, n, plan=plan), dtype=torch.uint8,
                           device=dev)
    else:
        temp = torch.empty(rs.rs_sort_u32(None, None, n, plan=plan), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        if wide_v64:
            rs.rs_sort_u64_pairs64(d_keys, d_vals, d_out, d_vout, n, 64, plan, temp, stream, want_offsets=True)
        elif vals64:
            rs.rs_sort_u32_pairs64(d_keys, d_vals, d_out, d_vout, n, 64, plan, temp, stream, want_offsets=True)
        elif wide and pairs:
            rs.rs_sort_u64_pairs(d_keys, d_vals, d_out, d_vout, n, 64, plan, temp, stream, want_offsets=True)
        elif wide:
            rs.rs_sort_u64(d_keys, d_out, n, 64, plan, temp, stream, want_offsets=True)
        elif pairs:
            rs.rs_sort_u32_pairs(d_keys, d_vals, d_out, d_vout, n, 64, plan, temp, stream, want_offsets=True)
        else:
            rs.rs_sort_u32(d_keys, d_out, n, 64, plan, temp, stream, want_offsets=True)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    rs.rs_trace_read()  # drop warm-up records

    # the timed steps; then the same steps again with every kernel bracketed
    # by CUDA events on its launching stream (the per-kernel times of the
    # roofline), kept apart because two event records per launch would
    # weigh on small sorts
    # inputs that fit in L2 are evicted before every timed step (a write of
    # a buffer larger than L2), and each step is timed on its own
    flush_l2 = 4 * n * (3 if vals64 else 2 if pairs else 1) * 2 < L2_BYTES
    flush_buf = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev) if flush_l2 else None
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # The clock record: nvidia-smi samples every 100 ms, and a timed region of
    # tens of milliseconds (a short --steps) may hold none.  So the sampler starts first, and
    # the same sort runs, untimed, for CLOCK_SETTLE_S before the timed steps;
    # the summary takes the samples from that start to the end of the traced
    # steps (all under this load) and counts those inside the timed region.
    with ClockSampler(local) as clocks:
        clocks.wait_first()
        load_t0 = time.monotonic()
        while time.monotonic() < load_t0 + CLOCK_SETTLE_S:
            step()
            torch.cuda.synchronize()
        barrier()
        timed_t0 = time.monotonic()
        if flush_l2:
            step_ms = 0.0
            for _ in range(args.steps):
                flush_buf.fill_(1)
                ev0.record(stream)
                step()
                ev1.record(stream)
                ev1.synchronize()
                step_ms += ev0.elapsed_time(ev1)
        else:
            ev0.record(stream)
            for _ in range(args.steps):
                step()
            ev1.record(stream)
        barrier()
        timed_t1 = time.monotonic()
        rs.rs_check_device_error()
        rs.rs_trace_enable(True)
        for _ in range(args.steps):
            step()
        barrier()
        rs.rs_trace_enable(False)
        load_t1 = time.monotonic()
    clock_summary = clocks.summary((load_t0, load_t1), (timed_t0, timed_t1))
    clock_summary["settle_s"] = CLOCK_SETTLE_S
    rs.rs_check_device_error()
    trace = rs.rs_trace_read()
    ms = max_over_ranks(step_ms if flush_l2 else ev0.elapsed_time(ev1), world, dev)
    ms_per_step = ms / args.steps
    value = whole_job_rate(n, world, args.steps, ms)

    # bytes of the executed plan: one read for the histograms, then a read
    # and a write per pass (keys; plus payload for pairs)
    pass_kind = None
    for k in ("onesweep_r11", "onesweep_r8"):
        if k in trace:
            pass_kind = k
    passes = trace[pass_kind]["launches"] // args.steps if pass_kind else 0
    # per key and pass: read + write of the words moved
    word_bytes = 8 * ((2 if wide else 1) + (2 if vals64 else 1 if pairs else 0))
    # 64-bit keys: the histograms read the interleaved keys once; where the
    # words are split into planes first, the split and the join (8 B read +
    # 8 B written each) come first and the histograms read each plane.
    # 64-bit values that are split and joined add the same 32 B.
    split = "split64" in trace
    if wide:
        # 64-bit values: the passes carry an index; the last one reads each
        # value (8 B) and writes it (8 B)
        bpk = (32 + 8 if split else 8) + passes * word_bytes + (16 if wide_v64 else 0)
    else:
        bpk = (32 if split else 0) + 4 + passes * word_bytes
    peak, peak_kind = measured_peak()
    roof = None
    msd = args.mode == "msd" and not wide and not vals64
    if msd:
        # MSD plan, every bucket within the local sort (uniform keys): keys
        # only: count read 4 + distribution 8 + local sort 8 = 20 B/key;
        # key+value: LSD histograms 4 + two stable passes 2 x 16 + count 4 +
        # local sort 16 = 56 B/key.  The roofline kernel is the one with the
        # most time per sort, against its own algorithmic bytes per sort.
        bpk = 56 if pairs else 20
        per_sort = {"msd_count": 4 * n, "msd_scatter": 8 * n, "local_sort": (16 if pairs else 8) * n,
                    "onesweep_r8": 2 * 16 * n, "upfront_hist": 4 * n}
        kind = max((k for k in trace if k in per_sort), key=lambda k: trace[k]["total_ms"], default=None)
        if kind:
            k_ms = trace[kind]["total_ms"] / args.steps
            achieved = per_sort[kind] / (k_ms * 1e-3) / 1e9
            roof = {"bound": "hbm", "kernel": kind, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                    "algorithmic_bytes_per_sort": per_sort[kind], "ms_per_sort": k_ms,
                    "launches_per_sort": trace[kind]["launches"] / args.steps}
        passes = 0
    if pass_kind and not msd:
        tr = trace[pass_kind]
        avg_ms = tr["total_ms"] / tr["launches"]
        bytes_launch = word_bytes * tr["keys"] / tr["launches"]
        achieved = bytes_launch / (avg_ms * 1e-3) / 1e9
        key = (f"{pass_kind}_{('keys64v64' if wide_v64 else 'keys64') if wide else ('pairs64' if vals64 else 'pairs' if pairs else 'keys')}"
               f"_n{n}")
        traffic = traffic_from_profiles(key)
        roof = {"bound": "hbm", "kernel": pass_kind, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": avg_ms}
        # The resource that binds the pass: shared-memory wavefronts (one per SM
        # per cycle at most).  Wavefronts per launch come from the same ncu
        # capture as the traffic; the rate uses this run's launch time and SM clock.
        waves = traffic_from_profiles(key + "_smem_wavefronts")
        if waves:
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            csum = clock_summary
            mhz = csum.get("sm_mhz") or csum.get("sm_max_mhz") or 2070.0
            per_cycle = waves / (avg_ms * 1e-3 * mhz * 1e6 * sms)
            roof["smem"] = {"wavefronts_per_launch": waves, "achieved_per_sm_cycle": per_cycle,
                            "peak_per_sm_cycle": 1.0, "frac": per_cycle, "sm_mhz": mhz, "sms": sms}
    launches = sum(v["launches"] for k, v in trace.items() if k != "clear")

    # end to end through the C entry for host buffers (rs_sort_u32_host):
    # pinned host keys (and values) in, sorted host arrays out, every copy
    # inside the timed region.  Consecutive sorts go round-robin to E2E_STREAMS
    # streams, each with its own device buffers, so that one sort's
    # device-to-host copy overlaps the next one's host-to-device copy and sort
    # (the host link carries both directions at once).  The one-stream figure
    # (copy in, sort, copy out, strictly one after another) is reported beside.
    e2e = None
    if not args.no_e2e and not wide and not vals64:
        h_in = torch.from_numpy(keys.view(np.int32)).pin_memory()
        h_vin = torch.arange(n, dtype=torch.int32).pin_memory() if pairs else None
        nb = rs.rs_sort_u32_host(None, h_vin, None, h_vin, n, plan=plan)
        streams = [torch.cuda.Stream(dev) for _ in range(E2E_STREAMS)]
        slots = []
        for _ in range(E2E_STREAMS):
            slots.append((torch.empty(nb, dtype=torch.uint8, device=dev), torch.empty_like(h_in).pin_memory(),
                          torch.empty_like(h_vin).pin_memory() if pairs else None))

        def e2e_run(steps, k):
            for i in range(steps):
                tmp, h_out, h_vout = slots[i % k]
                rs.rs_sort_u32_host(h_in, h_vin, h_out, h_vout, n, 64, plan, tmp, streams[i % k])

        def e2e_time(k):
            # CUDA events: the start is recorded on the current stream and
            # every copy stream waits on it; the end waits on every stream
            e2e_run(3, k)
            barrier()
            cur = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            for st in streams[:k]:
                st.wait_event(e0)
            e2e_run(args.steps, k)
            for st in streams[:k]:
                done = torch.cuda.Event()
                done.record(st)
                cur.wait_event(done)
            e1.record(cur)
            barrier()
            return whole_job_rate(n, world, args.steps, max_over_ranks(e0.elapsed_time(e1), world, dev))

        # the host link is shared with the machine's other work and its rate
        # varies from run to run: the piped figure is the median of three
        # measurements (all three are reported)
        serial = e2e_time(1)
        piped_runs = [e2e_time(E2E_STREAMS) for _ in range(3)]
        piped = statistics.median(piped_runs)
        rs.rs_check_device_error()
        per_step = (8 if pairs else 4) * n

        # The host link's own ceiling in this run: a step's copies in both
        # directions at once (the same pinned buffers and byte counts, no
        # sort), so that the end-to-end figure can be read against it.
        def link_rate(reps=10):
            src = [torch.zeros(n, dtype=torch.int32, device=dev) for _ in range(2 if pairs else 1)]
            dst = [torch.zeros(n, dtype=torch.int32, device=dev) for _ in range(2 if pairs else 1)]
            hin = [h_in] + ([h_vin] if pairs else [])
            hout = [slots[0][1]] + ([slots[0][2]] if pairs else [])
            cur = torch.cuda.current_stream()

            def timed(k):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(cur)
                for st in streams[:2]:
                    st.wait_event(e0)
                for _ in range(k):
                    with torch.cuda.stream(streams[0]):
                        for d, h in zip(dst, hin):
                            d.copy_(h, non_blocking=True)
                    with torch.cuda.stream(streams[1]):
                        for h, d in zip(hout, src):
                            h.copy_(d, non_blocking=True)
                for st in streams[:2]:
                    done = torch.cuda.Event()
                    done.record(st)
                    cur.wait_event(done)
                e1.record(cur)
                torch.cuda.synchronize()
                return e0.elapsed_time(e1) / k

            timed(3)  # warm-up
            ms = min(timed(reps) for _ in range(2))
            return {"value": n / ms / 1e6, "unit": "Gkeys/s", "ms_per_step": ms,
                    "gb_per_s_both_directions": 2 * per_step / ms / 1e6}

        for tmp, h_out, h_vout in slots:
            ok = np.array_equal(h_out.numpy().view(np.uint32)[:: max(1, n // 4096)],
                                sorted_by_kind(keys, args.key_kind)[:: max(1, n // 4096)])
            if not ok:
                raise SystemExit("end-to-end output is not the sorted keys")
        link = link_rate()  # after the check: it overwrites slot 0's host output
        link["frac"] = piped / link["value"]
        e2e = {"value": piped, "unit": "Gkeys/s", "h2d_bytes_per_step": per_step, "d2h_bytes_per_step": per_step,
               "streams": E2E_STREAMS, "repeats": piped_runs, "one_stream_value": serial,
               "api": "rs_sort_u32_host (pinned host buffers; copies of consecutive sorts overlap)",
               "link_ceiling": link}

    cpu = cpu_par = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(key_kind="u64" if wide else args.key_kind)
        if not wide and args.key_kind == "u32" and n == N_KEYS:
            cpu_par = cpu_parallel_baseline()

    # Beside the headline (the plain keys-only workload at 1 GPU): the same
    # keys with a payload, the batched form (config 4) and the served form
    # (config 5), each against its per-request plain launches.
    extra = {}
    headline = (world == 1 and not wide and not vals64 and not pairs and args.key_kind == "u32" and n == N_KEYS
                and not args.digit_bits and not args.tile and args.mode == "auto")
    if rank == 0 and headline and not args.no_extra:
        extra["pairs"] = measure_pairs(d_keys, args.steps, peak)
        del d_out, temp
        torch.cuda.empty_cache()
        extra["batched"] = measure_batched(args.steps, args.warmup)
        extra["served"] = served

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64" if wide else "u32", "data": "synthetic",
            "config": {"workload": (workload_label(n, pairs, args.key_kind).replace("key+payload", "key+64-bit value")
                                    if vals64 else workload_label(n, pairs, args.key_kind) if not wide else
                                    workload_label(n, pairs).replace("uint32 keys uniform in [0, 2^31-1]",
                                                                     "uint64 keys uniform over all 2^64 values")
                                    .replace("key+payload", "key+64-bit value" if wide_v64 else "key+payload")),
                       "n": n, "digit_bits": args.digit_bits or "auto", "mode": args.mode, "passes": passes,
                       "algorithmic_bytes_per_key": bpk,
                       "sort_roofline_frac": value / world * 1e9 * bpk / (peak * 1e9),
                       "l2": (f"inputs ({4 * n / 1e6:.0f} MB) exceed L2 ({L2_BYTES / 1e6:.0f} MB); no flush"
                              if not flush_l2 else
                              f"inputs ({4 * n / 1e6:.1f} MB) fit in L2: a {FLUSH_BYTES >> 20} MiB buffer is written "
                              "before every timed step, outside its events"),
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "cpu_parallel_baseline": cpu_par,
            "e2e": e2e,
            "gpu_launches": launches,
            "kernel_ms": {k: v["total_ms"] / max(v["launches"], 1) for k, v in trace.items()},
            "kernel_ms_per_step": {k: v["total_ms"] / args.steps for k, v in trace.items()},
            "clocks": clock_summary,
            **extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ------------------------------------------------------- other workloads
def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def measure_pairs(d_keys, steps: int, peak: float) -> dict:
    """The headline keys with a uint32 payload (payload = input position):
    whole-sort rate, the pass kernel's time and its fraction of the HBM
    peak at 16 algorithmic bytes per key (8 read, 8 written)."""
    import torch
    import paper_cs_0004013_gb300 as rs
    n = d_keys.numel()
    d_vals = torch.arange(n, dtype=torch.int32, device=d_keys.device)
    ko, vo = torch.empty_like(d_keys), torch.empty_like(d_vals)
    temp = torch.empty(rs.rs_sort_u32_pairs(None, None, None, None, n), dtype=torch.uint8, device=d_keys.device)
    for _ in range(3):
        rs.rs_sort_u32_pairs(d_keys, d_vals, ko, vo, n, 64, None, temp)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    idx = torch.arange(0, n, max(1, n // 4096), device=d_keys.device)
    if not torch.equal(d_keys[vo[idx].long()], ko[idx]):
        raise SystemExit("key+payload output: payloads do not carry their keys")
    rs.rs_trace_read()
    rs.rs_trace_enable(True)
    e0, e1 = _events()
    e0.record()
    for _ in range(steps):
        rs.rs_sort_u32_pairs(d_keys, d_vals, ko, vo, n, 64, None, temp)
    e1.record()
    torch.cuda.synchronize()
    rs.rs_trace_enable(False)
    trace = rs.rs_trace_read()
    ms = e0.elapsed_time(e1) / steps
    p = trace.get("onesweep_r8", {})
    pass_ms = p["total_ms"] / p["launches"] if p else None
    value = n / (ms * 1e-3) / 1e9
    out = {"value": value, "unit": "Gkeys/s", "ms_per_step": ms, "steps": steps,
           "workload": workload_label(n, True), "algorithmic_bytes_per_key": 68,
           "sort_roofline_frac": value * 1e9 * 68 / (peak * 1e9)}
    if pass_ms:
        out["pass"] = {"kernel": "onesweep_r8", "avg_launch_ms": pass_ms,
                       "frac": 16 * n / (pass_ms * 1e-3) / (peak * 1e9),
                       "traffic": traffic_from_profiles(f"onesweep_r8_pairs_n{n}")}
    del ko, vo, temp, d_vals
    return out


def measure_batched(steps: int, warmup: int) -> dict:
    """Config 4: up to 4096 key+payload arrays, sizes log-uniform in
    [2^10, 2^20], drawn until 2^28 keys; one rs_sort_u32_segmented call
    (also replayed from a CUDA graph) vs one rs_sort_u32_pairs call per array."""
    import torch
    import synth
    import paper_cs_0004013_gb300 as rs
    keys, vals, offs = synth.segmented_batch(synth.CONFIG_SEED + 4)
    n, S = keys.size, offs.size - 1
    dk = torch.from_numpy(keys.view(np.int32)).cuda()
    dv = torch.from_numpy(vals.view(np.int32)).cuda()
    ko, vo = torch.empty_like(dk), torch.empty_like(dv)
    d_off = torch.from_numpy(offs.view(np.int64)).cuda()
    d_po = torch.empty(S * 65, dtype=torch.int64, device="cuda")
    temp = torch.empty(rs.rs_sort_u32_segmented(None, dv, None, vo, None, offs, S, n, 64), dtype=torch.uint8,
                       device="cuda")
    stream = torch.cuda.current_stream()

    # The autotuner times the segmented plans on this batch and installs the
    # winner for its size class; the timed call passes no plan, so it runs
    # the tuned one.  The compiled default is timed beside it.
    from paper_cs_0004013_gb300 import tune
    import tempfile
    tuner = tune.Tuner(cache_path=os.path.join(tempfile.mkdtemp(), "plans.json"), reps=2)
    tuned = tuner.best_segmented_plan(offs, pairs=True, keys=dk, vals=dv)
    tuner.install()
    default_plan = {"digit_bits": 8, "mode": 0, "tile": 3}  # the compiled default
    temp = torch.empty(max(temp.numel(), rs.rs_sort_u32_segmented(None, dv, None, vo, None, offs, S, n, 64)),
                       dtype=torch.uint8, device="cuda")

    def batched(plan=None):
        rs.rs_sort_u32_segmented(dk, dv, ko, vo, d_off, offs, S, n, 64, d_po, plan, temp, stream)

    for _ in range(max(warmup, 3)):
        batched()
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    # correctness spot check against numpy on a few segments
    for s_ in (0, S // 2, S - 1):
        a, b = int(offs[s_]), int(offs[s_ + 1])
        got = ko[a:b].cpu().numpy().view(np.uint32)
        if not np.array_equal(got, np.sort(keys[a:b])):
            raise SystemExit(f"batched output wrong in segment {s_}")
    rs.rs_trace_read()
    rs.rs_trace_enable(True)
    e0, e1 = _events()
    e0.record(stream)
    for _ in range(steps):
        batched()
    e1.record(stream)
    torch.cuda.synchronize()
    rs.rs_trace_enable(False)
    trace = rs.rs_trace_read()
    t_batched = e0.elapsed_time(e1) / steps
    batched(default_plan)
    e0.record(stream)
    for _ in range(steps):
        batched(default_plan)
    e1.record(stream)
    torch.cuda.synchronize()
    t_default = e0.elapsed_time(e1) / steps
    # the same work captured once into a CUDA graph and replayed
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        batched()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        rs.rs_sort_u32_segmented(dk, dv, ko, vo, d_off, offs, S, n, 64, d_po, None, temp, side)
    g.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    t_graph = e0.elapsed_time(e1) / steps
    # one plain call per array
    big = int(np.diff(offs).max())
    ptemp = torch.empty(rs.rs_sort_u32_pairs(None, None, None, None, big), dtype=torch.uint8, device="cuda")

    def per_array():
        for s_ in range(S):
            a, b = int(offs[s_]), int(offs[s_ + 1])
            rs.rs_sort_u32_pairs(dk[a:b], dv[a:b], ko[a:b], vo[a:b], b - a, 64, None, ptemp, stream,
                                 want_offsets=True)

    per_array()
    torch.cuda.synchronize()
    reps = max(1, steps // 5)
    e0.record(stream)
    for _ in range(reps):
        per_array()
    e1.record(stream)
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / reps
    rs.rs_check_device_error()
    cls = tune.size_log2(-(-n // S))
    rs.rs_set_default_plan(rs.RS_ENTRY_SEGMENTED_PAIRS, cls, None)
    del dk, dv, ko, vo, temp, ptemp
    torch.cuda.empty_cache()
    return {"value": n / (t_batched * 1e-3) / 1e9, "unit": "Gkeys/s", "ms_per_step": t_batched,
            "tuned_plan": tuned, "size_class": cls,
            "default_plan": {"plan": default_plan, "value": n / (t_default * 1e-3) / 1e9, "unit": "Gkeys/s",
                             "ms_per_step": t_default},
            "steps": steps, "workload": f"batched segmented sort: {S} key+payload arrays, log-uniform sizes in "
                                        f"[2^10, 2^20], {n} keys in total, one rs_sort_u32_segmented call",
            "segments": int(S), "n": int(n),
            "graph_replay": {"value": n / (t_graph * 1e-3) / 1e9, "unit": "Gkeys/s", "ms_per_step": t_graph},
            "per_array_plain": {"value": n / (t_plain * 1e-3) / 1e9, "unit": "Gkeys/s", "ms_per_step": t_plain,
                                "calls_per_step": int(S), "steps": reps},
            "speedup_vs_per_array": t_plain / t_batched,
            "kernel_ms": {k: v["total_ms"] / v["launches"] for k, v in trace.items()}}


def run_batched(args):
    import torch
    torch.cuda.set_device(0)
    b = measure_batched(args.steps, args.warmup)
    line = {"metric": METRIC, "value": b["value"], "unit": "Gkeys/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": b["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": b["workload"], "segments": b["segments"], "n": b["n"]},
            **{k: b[k] for k in ("tuned_plan", "default_plan", "graph_replay", "per_array_plain",
                                 "speedup_vs_per_array", "kernel_ms")}}
    print(json.dumps(line), flush=True)
    return 0


SERVE_POOL_KEYS = 1 << 27


def measure_served(requests: int, rounds: int) -> dict:
    """Config 5: Poisson arrivals of sorts with sizes log-uniform in
    [2^16, 2^26] (keys-only or pairs with probability 1/2), served with
    continuous batching at 0.5x, 0.8x and 1.2x the measured serial capacity;
    p50/p99 latency (arrival -> result on the host) and sustained keys/s.
    Each request's keys are a slice of one pinned pool of 2^27 seeded keys
    (at a per-request offset) and its payload the input positions; results
    land in pinned buffers the server lends from a result pool, so that a
    thousand requests per point fit in host memory.  After the timed runs, an
    untimed run checks every 50th result against numpy's sort."""
    import torch
    import synth
    import paper_cs_0004013_gb300 as rs
    from paper_cs_0004013_gb300.serve import Request, ResultPool, SortServer, latency_stats, serial_plain
    pool_k = torch.from_numpy(synth.uniform31(SERVE_POOL_KEYS, synth.CONFIG_SEED + 5).view(np.int32)).pin_memory()
    pool_v = torch.arange(1 << 26, dtype=torch.int32).pin_memory()
    checked = {"n": 0, "bad": 0}

    def make(rate, seed):
        out = []
        for q in synth.serving_requests(requests, seed, rate_per_s=rate):
            off = int(q["seed"] % (SERVE_POOL_KEYS - q["n"]))
            k = pool_k[off: off + q["n"]]
            v = pool_v[: q["n"]] if q["pairs"] else None
            out.append(Request.view(q["id"], q["arrival_s"], k, v))
        return out

    def on_done(r):
        if r.id % 50 == 0 and r.error is None:
            checked["n"] += 1
            if not np.array_equal(r.out_keys.numpy().view(np.uint32), np.sort(r.keys.numpy().view(np.uint32))):
                checked["bad"] += 1

    base = make(1.0, synth.CONFIG_SEED + 5)
    total_keys = sum(r.n for r in base)
    serial_plain(base[:20])  # warm-up
    t_serial = serial_plain(base)
    serial_rate = total_keys / t_serial / 1e9
    cap_req_s = len(base) / t_serial
    # sixteen batches in flight on sixteen streams (closed loop on GB300:
    # 21.5-22.0 Gkeys/s against 19.4 with eight); results lent from a 16 GiB
    # pinned pool
    srv = SortServer(slots=16, streams=16, mem_budget=24 << 30, result_pool=ResultPool(16 << 30))
    # warm-up: one whole closed-loop run, so that the device pools and the
    # pinned result pool hold every size class the timed runs need
    srv.run(make(1e9, synth.CONFIG_SEED + 5), realtime=False)
    points = []
    for load in (0.5, 0.8, 1.2):
        reqs = make(cap_req_s * load, synth.CONFIG_SEED + 5)
        srv.run(reqs, realtime=True)
        rs.rs_check_device_error()
        span = max(r.done_s for r in reqs) - min(r.arrival_s for r in reqs)
        st = latency_stats(reqs)
        st.update({"offered_load": load, "requests": len(reqs), "sustained_gkeys_s": total_keys / span / 1e9,
                   "batches": len({r.batch for r in reqs}), "failed": sum(r.error is not None for r in reqs)})
        points.append(st)
    # closed loop: everything arrives at once
    t_closed = []
    for _ in range(max(rounds, 1)):
        reqs = make(1e9, synth.CONFIG_SEED + 5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        srv.run(reqs, realtime=False)
        t_closed.append(time.perf_counter() - t0)
    t_closed = statistics.median(t_closed)
    # an untimed closed-loop run that checks every 50th result when it completes
    srv.on_done = on_done
    srv.run(make(1e9, synth.CONFIG_SEED + 5), realtime=False)
    srv.on_done = None
    if checked["bad"] or srv.failed:
        raise SystemExit(f"served results wrong: {checked['bad']} of {checked['n']} checked, {srv.failed} failed")
    return {"value": total_keys / t_closed / 1e9, "unit": "Gkeys/s", "seconds": t_closed,
            "workload": f"serving: {len(base)} requests, sizes log-uniform in [2^16, 2^26], half key+payload; "
                        "value = closed-loop keys/s including host<->device copies",
            "requests": len(base), "total_keys": int(total_keys),
            "serial_plain": {"value": serial_rate, "unit": "Gkeys/s", "seconds": t_serial},
            "speedup_vs_serial": (total_keys / t_closed / 1e9) / serial_rate,
            "load_points": points, "results_checked": checked["n"]}


def measure_served_in_own_process(requests: int) -> dict:
    """The served form measured by `bench.py --workload serve` in a process
    of its own, as a server would run, started before the bench's own
    process touches the GPU.  Run inside the bench's process after the other
    measurements, or in a child while that process held its GPU context and
    buffers, the same loop ran about a fifth slower with p99 latencies four
    times longer, and so did the serial baseline beside it."""
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", "serve", "--steps", "50",
           "--requests", str(requests)]
    res = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT)
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    if res.returncode != 0 or not lines:
        raise SystemExit(f"served measurement failed (rc {res.returncode}): {res.stderr[-2000:]}")
    d = json.loads(lines[-1])
    return {"value": d["value"], "unit": d["unit"], "seconds": d["ms_per_step"] / 1e3,
            "workload": d["config"]["workload"], "requests": requests, "total_keys": d["config"]["total_keys"],
            "serial_plain": d["serial_plain"], "speedup_vs_serial": d["speedup_vs_serial"],
            "load_points": d["load_points"], "results_checked": d["results_checked"],
            "rounds": d["steps"], "process": "own (bench.py --workload serve)"}


def run_serve(args):
    import torch
    torch.cuda.set_device(0)
    rounds = min(max(args.steps // 10, 1), 5)
    sv = measure_served(args.requests, rounds)
    line = {"metric": METRIC, "value": sv["value"], "unit": "Gkeys/s", "n_gpus": 1,
            "steps": rounds, "warmup": 1, "ms_per_step": sv["seconds"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": sv["workload"], "total_keys": sv["total_keys"]},
            **{k: sv[k] for k in ("serial_plain", "speedup_vs_serial", "load_points", "results_checked")}}
    print(json.dumps(line), flush=True)
    return 0


def run_dist(args):
    """Config 3: 2^26 keys in the four skewed distributions, keys only."""
    import torch
    import synth
    import paper_cs_0004013_gb300 as rs
    torch.cuda.set_device(0)
    res = {}
    for dist in ("skewed_chunks", "few_distinct", "gauss_mix", "tight_clusters"):
        keys = synth.config_keys(3, dist=dist)
        d = torch.from_numpy(keys.view(np.int32)).cuda()
        out = torch.empty_like(d)
        temp = torch.empty(rs.rs_sort_u32(None, None, d.numel()), dtype=torch.uint8, device="cuda")
        for _ in range(3):
            rs.rs_sort_u32(d, out, d.numel(), 64, None, temp)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        for _ in range(args.steps):
            rs.rs_sort_u32(d, out, d.numel(), 64, None, temp)
        e1.record()
        torch.cuda.synchronize()
        rs.rs_check_device_error()
        ms = e0.elapsed_time(e1) / args.steps
        res[dist] = {"gkeys_s": d.numel() / ms / 1e6, "ms": ms}
    line = {"metric": METRIC, "value": min(v["gkeys_s"] for v in res.values()), "unit": "Gkeys/s",
            "n_gpus": 1, "steps": args.steps, "warmup": 3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "2^26 keys, four skewed distributions, keys only; value = the slowest"},
            "per_distribution": res}
    print(json.dumps(line), flush=True)
    return 0


def run_merge(args):
    """NEXT-4: stable merge of two sorted runs of 2^26 uniform 31-bit keys
    (the runs sorted by the library first), keys only and with payloads;
    value = merged keys per second (keys only)."""
    import torch
    import synth
    import paper_cs_0004013_gb300 as rs
    torch.cuda.set_device(0)
    n = args.n
    runs = []
    for seed in (synth.CONFIG_SEED + 41, synth.CONFIG_SEED + 42):
        d = torch.from_numpy(synth.uniform31(n, seed).view(np.int32)).cuda()
        runs.append(rs.sort(d)[0])
    a, b = runs
    peak, peak_kind = measured_peak()
    res = {}
    for pairs in (False, True):
        va = torch.arange(n, dtype=torch.int32, device="cuda") if pairs else None
        vb = torch.arange(n, 2 * n, dtype=torch.int32, device="cuda") if pairs else None
        out = torch.empty(2 * n, dtype=torch.int32, device="cuda")
        vout = torch.empty_like(out) if pairs else None
        temp = torch.empty(rs.rs_merge_u32(None, va, n, None, vb, n, None, vout), dtype=torch.uint8, device="cuda")

        def step():
            rs.rs_merge_u32(a, va, n, b, vb, n, out, vout, 64, None, temp, want_offsets=True)

        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        rs.rs_check_device_error()
        ms = e0.elapsed_time(e1) / args.steps
        bytes_per_key = 16 if pairs else 8  # read once, written once
        gbs = 2 * n * bytes_per_key / (ms * 1e-3) / 1e9
        res["pairs" if pairs else "keys"] = {"gkeys_s": 2 * n / ms / 1e6, "ms": ms, "achieved_gbs": gbs,
                                             "frac": gbs / peak}
    sample = slice(None, None, max(1, n // 2048))
    merged = out.cpu().numpy().view(np.uint32)
    if not np.all(merged[sample][1:] >= merged[sample][:-1]):
        raise SystemExit("merged output is not ascending")
    line = {"metric": METRIC, "value": res["keys"]["gkeys_s"], "unit": "Gkeys/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": res["keys"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"stable merge of two sorted runs of {n} uniform 31-bit keys; value = merged "
                                   "keys per second, keys only", "n_per_run": n},
            "roofline": {"bound": "hbm", "kernel": "merge", "achieved": res["keys"]["achieved_gbs"], "peak": peak,
                         "unit": "GB/s", "frac": res["keys"]["frac"], "traffic": None, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_key": 8},
            "with_payloads": res["pairs"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "dist":
        return run_dist(args)
    if args.workload == "merge":
        return run_merge(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
