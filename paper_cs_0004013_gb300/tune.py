"""Plan autotuner: picks the digit width (8 or 11 bits), LSD or MSD, and the
tile shape per size class and payload flag by timing the candidates on the
GPU in use, remembers the winners, and installs them in the library so
that calls made without a plan (the plain sorts, the segmented sort, the
serving loop) run them.

The paper chose its algorithm per data set by measurement as well (Sec. 4.2:
the bucketing + local radix pipeline for four data sets, a different one
for the clustered fifth); here the measurement is automated per size class.

Results are cached in a JSON file keyed by GPU name, entry kind (plain or
segmented), size class (ceil(log2) of n, or of the mean segment size for a
segmented batch), payload flag and an optional distribution label.  Timing
uses CUDA events on the current stream; every candidate runs through the
same C entry points as a user's call, so the tuner measures exactly what it
will select.  `install()` hands the cached winners of this GPU to the
library (rs_set_default_plan), where they apply to calls whose plan is NULL
or leaves fields zero.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

__all__ = ["Tuner", "candidate_plans", "segmented_candidates", "size_class", "size_log2"]

RS_MODE_AUTO, RS_MODE_LSD, RS_MODE_MSD = 0, 1, 2
# rs_set_default_plan entries
ENTRY = {("plain", False): 0, ("plain", True): 1, ("segmented", False): 2, ("segmented", True): 3}


def size_log2(n: int) -> int:
    """ceil(log2(n)) (0 for n <= 1): the library's size class."""
    return max(0, math.ceil(math.log2(max(n, 1))))


def size_class(n: int) -> int:
    return 1 << size_log2(n)


def candidate_plans(n: int, pairs: bool) -> list[dict]:
    """Plans worth timing for a plain sort of n keys: the automatic plan
    (which sorts up to 16,384 keys in one block), 8-bit LSD over its tile
    shapes (lane-mask and half-warp-group kernels), 11-bit LSD over its
    large tiles, and the MSD plan where its buckets can fit the local sort."""
    out = [{"digit_bits": 0, "mode": RS_MODE_AUTO, "tile": 0}]
    out += [{"digit_bits": 8, "mode": RS_MODE_LSD, "tile": t} for t in (1, 2, 3, 5, 6, 7, 8)]
    out += [{"digit_bits": 11, "mode": RS_MODE_LSD, "tile": t} for t in (2, 4)]
    if n < (1 << 30) - (1 << 16):
        out.append({"digit_bits": 8, "mode": RS_MODE_MSD, "tile": 0})
    return out


def segmented_candidates(pairs: bool) -> list[dict]:
    """Plans of the segmented sort: its three tiled-pass shapes, each with the
    one-block local sort for every segment that fits (MSD: bucket, then
    local sort) or only for the smallest class (LSD: tiled passes above
    4,096 keys)."""
    return [{"digit_bits": 8, "mode": m, "tile": t} for t in (1, 2, 3) for m in (RS_MODE_MSD, RS_MODE_LSD)]


def _default_cache() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "rsort_gb300", "plans.json")


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


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
    def key(gpu: str, n: int, pairs: bool, dist: str, kind: str = "plain") -> str:
        """Cache key; n is the keys of a plain sort or the mean segment size."""
        return f"{gpu}|{kind}|{size_log2(n)}|{'pairs' if pairs else 'keys'}|{dist}"

    @staticmethod
    def _gpu(gpu):
        if gpu is None:
            import torch
            gpu = torch.cuda.get_device_name()
        return gpu

    # -- timing
    def _time(self, run) -> float:
        import torch
        import paper_cs_0004013_gb300 as rs
        run()
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        for _ in range(self.reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        rs.rs_check_device_error()
        return e0.elapsed_time(e1) / self.reps

    def time_plan(self, plan: dict, keys, vals=None) -> float:
        """Milliseconds per plain sort of `keys` (CUDA tensor) under `plan`,
        or inf if the plan is not available for this size."""
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

        return self._time(run)

    def time_segmented(self, plan: dict, keys, vals, h_offs) -> float:
        """Milliseconds per segmented sort of the batch (keys / vals CUDA
        tensors, h_offs numpy uint64 offsets) under `plan`, or inf."""
        import torch
        import paper_cs_0004013_gb300 as rs
        S, n = h_offs.size - 1, int(h_offs[-1])
        try:
            nb = rs.rs_sort_u32_segmented(None, vals, None, vals, None, h_offs, S, n, 64, plan=plan)
        except rs.RsError:
            return math.inf
        temp = torch.empty(nb, dtype=torch.uint8, device=keys.device)
        d_off = torch.from_numpy(h_offs.view(np.int64)).to(keys.device)
        out = torch.empty_like(keys)
        vout = None if vals is None else torch.empty_like(vals)

        def run():
            rs.rs_sort_u32_segmented(keys, vals, out, vout, d_off, h_offs, S, n, 64, None, plan, temp)

        return self._time(run)

    def _pick(self, k: str, timings: list) -> dict:
        ms, plan = min(timings, key=lambda x: x[0])
        cache = self._load()
        cache[k] = {"plan": plan, "ms": ms,
                    "timings": [{"plan": p, "ms": (None if math.isinf(t) else t)} for t, p in timings]}
        self._save()
        return dict(plan)

    def best_plan(self, n: int, pairs: bool = False, dist: str = "uniform", keys=None, vals=None,
                  gpu: str | None = None) -> dict:
        """The fastest plain-sort candidate for this size class (cached).
        Times on `keys` / `vals` when given, else on seeded uniform 31-bit keys."""
        gpu = self._gpu(gpu)
        k = self.key(gpu, n, pairs, dist)
        cache = self._load()
        if k in cache:
            return dict(cache[k]["plan"])
        if keys is None:
            import torch
            g = torch.Generator(device="cuda").manual_seed(12345)
            keys = torch.randint(0, 1 << 31, (n,), generator=g, dtype=torch.int64, device="cuda").to(torch.int32)
            vals = torch.arange(n, dtype=torch.int32, device="cuda") if pairs else None
        return self._pick(k, [(self.time_plan(p, keys, vals), p) for p in candidate_plans(n, pairs)])

    def best_segmented_plan(self, h_offs, pairs: bool = False, dist: str = "uniform", keys=None, vals=None,
                            gpu: str | None = None) -> dict:
        """The fastest segmented-sort candidate for the batch's size class
        (mean segment size; cached).  Times on the batch itself when keys
        (and vals) are given, else on seeded uniform 31-bit keys with the
        batch's segment offsets."""
        gpu = self._gpu(gpu)
        h_offs = np.asarray(h_offs, dtype=np.uint64)
        S, n = h_offs.size - 1, int(h_offs[-1])
        k = self.key(gpu, -(-n // max(S, 1)), pairs, dist, kind="segmented")
        cache = self._load()
        if k in cache:
            return dict(cache[k]["plan"])
        if keys is None:
            import torch
            g = torch.Generator(device="cuda").manual_seed(12345)
            keys = torch.randint(0, 1 << 31, (n,), generator=g, dtype=torch.int64, device="cuda").to(torch.int32)
            vals = torch.arange(n, dtype=torch.int32, device="cuda") if pairs else None
        return self._pick(k, [(self.time_segmented(p, keys, vals, h_offs), p) for p in segmented_candidates(pairs)])

    def install(self, gpu: str | None = None) -> int:
        """Hands every cached winner of this GPU (distribution "uniform") to
        the library, so that calls without a plan use it.  Returns how many
        were installed."""
        import paper_cs_0004013_gb300 as rs
        gpu = self._gpu(gpu)
        done = 0
        for k, v in self._load().items():
            parts = k.split("|")
            if len(parts) != 5 or parts[0] != gpu or parts[4] != "uniform":
                continue
            kind, cls, flag = parts[1], int(parts[2]), parts[3] == "pairs"
            if (kind, flag) not in ENTRY or not 0 <= cls <= 32:
                continue
            plan = {f: int(v["plan"].get(f, 0)) for f in ("digit_bits", "mode", "tile")}
            rs.rs_set_default_plan(ENTRY[(kind, flag)], cls, plan)
            done += 1
        return done
