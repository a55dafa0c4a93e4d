"""Plan autotuner: picks the digit width (8 or 11 bits), LSD or MSD, and the
tile shape for a size class and payload flag by timing the candidates on
the GPU in use, and remembers the winner.

The library's own defaults (compiled in) come from one such sweep at 2^26
keys; the tuner refines them per size class.  Results are cached in a JSON
file keyed by GPU name, size class (power of two above n), payload flag and
an optional distribution label.  Timing uses CUDA events on the current
stream; every candidate runs through the same C entry points as a user's
call, so the tuner measures exactly what it will select.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

__all__ = ["Tuner", "candidate_plans", "size_class"]

RS_MODE_LSD, RS_MODE_MSD = 1, 2


def size_class(n: int) -> int:
    return 1 << max(0, math.ceil(math.log2(max(n, 1))))


def candidate_plans(n: int, pairs: bool) -> list[dict]:
    """Plans worth timing for n keys: 8-bit LSD over its tile shapes
    (plain and persistent pipelined kernels), 11-bit LSD over its large
    tiles, and the MSD plan where its buckets can fit the local sort."""
    out = [{"digit_bits": 8, "mode": RS_MODE_LSD, "tile": t} for t in (1, 2, 3, 5, 6, 7)]
    out += [{"digit_bits": 11, "mode": RS_MODE_LSD, "tile": t} for t in (2, 4)]
    if n < (1 << 30) - (1 << 16):
        out.append({"digit_bits": 8, "mode": RS_MODE_MSD, "tile": 0})
    return out


def _default_cache() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "rsort_gb300", "plans.json")


class Tuner:
    def __init__(self, cache_path: str | None = None, reps: int = 3):
        self.cache_path = cache_path or _default_cache()
        self.reps = reps
        self._cache = None

    # -- cache
    def _load(self) -> dict:
        if self._cache is None:
            try:
                with open(self.cache_path) as f:
                    self._cache = json.load(f)
            except (OSError, ValueError):
                self._cache = {}
        return self._cache

    def _save(self) -> None:
        os.makedirs(os.path.dirname(self.cache_path), exist_ok=True)
        tmp = self.cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self._cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    @staticmethod
    def key(gpu: str, n: int, pairs: bool, dist: str) -> str:
        return f"{gpu}|{size_class(n)}|{'pairs' if pairs else 'keys'}|{dist}"

    # -- timing
    def time_plan(self, plan: dict, keys, vals=None) -> float:
        """Milliseconds per sort of `keys` (CUDA tensor) under `plan`, or inf
        if the plan is not available for this size."""
        import torch
        import paper_cs_0004013_gb300 as rs
        n = keys.numel()
        try:
            if vals is None:
                temp = torch.empty(rs.rs_sort_u32(None, None, n, plan=plan), dtype=torch.uint8, device=keys.device)
            else:
                temp = torch.empty(rs.rs_sort_u32_pairs(None, None, None, None, n, plan=plan), dtype=torch.uint8,
                                   device=keys.device)
        except rs.RsError:
            return math.inf
        out = torch.empty_like(keys)
        vout = None if vals is None else torch.empty_like(vals)

        def run():
            if vals is None:
                rs.rs_sort_u32(keys, out, n, 64, plan, temp, want_offsets=False)
            else:
                rs.rs_sort_u32_pairs(keys, vals, out, vout, n, 64, plan, temp, want_offsets=False)

        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(self.reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        rs.rs_check_device_error()
        return e0.elapsed_time(e1) / self.reps

    def best_plan(self, n: int, pairs: bool = False, dist: str = "uniform", keys=None, vals=None,
                  gpu: str | None = None) -> dict:
        """The fastest candidate plan for this size class (cached).  Times
        on `keys` / `vals` when given, else on seeded uniform 31-bit keys."""
        if gpu is None:
            import torch
            gpu = torch.cuda.get_device_name()
        k = self.key(gpu, n, pairs, dist)
        cache = self._load()
        if k in cache:
            return dict(cache[k]["plan"])
        if keys is None:
            import torch
            g = torch.Generator(device="cuda").manual_seed(12345)
            keys = torch.randint(0, 1 << 31, (n,), generator=g, dtype=torch.int64, device="cuda").to(torch.int32)
            vals = torch.arange(n, dtype=torch.int32, device="cuda") if pairs else None
        timings = []
        for plan in candidate_plans(n, pairs):
            timings.append((self.time_plan(plan, keys, vals), plan))
        ms, plan = min(timings, key=lambda x: x[0])
        cache[k] = {"plan": plan, "ms": ms,
                    "timings": [{"plan": p, "ms": (None if math.isinf(t) else t)} for t, p in timings]}
        self._save()
        return dict(plan)
