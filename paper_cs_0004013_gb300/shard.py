"""Sorting keys spread over several ranks: the paper's machine-level algorithm
(Sec. 3) with GPUs as cells.

Each rank holds a shard of uint32 keys (any sizes, empty included).  The
result: rank q holds positions [off[q], off[q+1]) of the globally sorted
keys, off being the equal-partition offsets of the contract (Sec. 1.1; the
lower ranks take the extra key when the rank count does not divide the total,
footnote 7 of Sec. 3.4.2).

1. Bucketing counts (Sec. 3.2): every rank counts its keys per bucket of the
   top bits (buckets = the keys' bits 22-31, 1024 of them; the paper used
   4096-8192 for 64 cells).
2. Global totals (Sec. 4.4 sums them over a hypercube): every rank gathers
   every rank's counts, which also gives each (rank, bucket) its exact place.
3. Bucket -> rank: bucket d goes to the rank whose output partition holds the
   bucket's first position, so each rank receives a contiguous bucket range.
4. Distribution (Sec. 3.2): each rank sorts its shard (the rank-local radix
   sort, so that its keys are grouped by destination in order) and sends each
   rank its slice in one all-to-all.
5. Local sort (Sec. 3.3): each rank sorts what it received.
6. Post-balance (Sec. 3.5): buckets do not end exactly on partition
   boundaries, so every rank sends the keys outside its exact partition to
   the ranks that own those positions (one more all-to-all; the counts are
   known to every rank from step 2, so nothing else is exchanged).

The rank-local steps (counting, sorting) run through an `ops` object: the
default uses librsort's kernels on the rank's GPU; the exchanges use
torch.distributed (NCCL with CUDA tensors; with gloo the keys are staged
through host memory).  No multicast and no peer loads: every exchange is a
collective of the process group.
"""
from __future__ import annotations

import numpy as np

__all__ = ["CudaOps", "sharded_sort", "bucket_destinations", "partition_offsets_of", "exchange_plan"]

BUCKET_SHIFT = 22  # buckets are the keys' bits 22-31
NUM_BUCKETS = 1 << (32 - BUCKET_SHIFT)


class CudaOps:
    """Rank-local steps on the rank's GPU through librsort."""

    def __init__(self, device):
        import torch
        self.device = torch.device(device)

    def bucket_counts(self, keys) -> np.ndarray:
        """Keys per bucket (bits 22-31): the top digit of the 11-bit plan's
        upfront histogram (digits of 11, 11 and 10 bits)."""
        import torch
        import paper_cs_0004013_gb300 as rs
        n = keys.numel()
        h = torch.zeros(3 * 2048, dtype=torch.int32, device=self.device)
        if n:
            rs.rs_digit_histograms(keys, n, 11, h)
        return h[2 * 2048: 2 * 2048 + NUM_BUCKETS].cpu().numpy().view(np.uint32).astype(np.int64)

    def sort(self, keys):
        import paper_cs_0004013_gb300 as rs
        if keys.numel() == 0:
            return keys
        out, _ = rs.sort(keys)
        return out

    def to_comm(self, x, backend: str):
        return x.cpu() if backend == "gloo" else x

    def from_comm(self, x, backend: str):
        return x.to(self.device) if backend == "gloo" else x

    def empty(self, n: int, backend: str):
        import torch
        return torch.empty(n, dtype=torch.int32, device="cpu" if backend == "gloo" else self.device)


def partition_offsets_of(total: int, parts: int) -> np.ndarray:
    """off[q] = q * floor(total / parts) + min(q, total mod parts)."""
    q, r = divmod(total, parts)
    return np.array([p * q + min(p, r) for p in range(parts + 1)], dtype=np.int64)


def bucket_destinations(totals: np.ndarray, parts: int) -> np.ndarray:
    """Rank of each bucket: the one whose output partition holds the bucket's
    first position (empty buckets follow their predecessor's rank)."""
    total = int(totals.sum())
    off = partition_offsets_of(total, parts)
    start = np.concatenate([[0], np.cumsum(totals)[:-1]])
    dest = np.searchsorted(off[1:], start, side="right")
    return np.minimum(dest, parts - 1).astype(np.int64)


def exchange_plan(counts: np.ndarray) -> dict:
    """Everything the exchanges need, from the gathered per-rank bucket counts
    (counts[r][d]): what each rank sends to each rank in the distribution
    (send[r][q]), what each rank holds after it (held[q]), and the post-balance
    moves (move[q][t]: keys rank q sends to rank t so that every rank ends
    with its exact partition)."""
    P = counts.shape[0]
    totals = counts.sum(axis=0)
    dest = bucket_destinations(totals, P)
    send = np.zeros((P, P), dtype=np.int64)
    for q in range(P):
        send[:, q] = counts[:, dest == q].sum(axis=1)
    held = send.sum(axis=0)
    total = int(totals.sum())
    off = partition_offsets_of(total, P)
    held_start = np.concatenate([[0], np.cumsum(held)[:-1]])
    move = np.zeros((P, P), dtype=np.int64)
    for q in range(P):  # rank q holds global positions [held_start[q], held_start[q] + held[q])
        lo, hi = int(held_start[q]), int(held_start[q] + held[q])
        for t in range(P):  # rank t must end with positions [off[t], off[t+1])
            a, b = max(lo, int(off[t])), min(hi, int(off[t + 1]))
            move[q, t] = max(0, b - a)
    return {"dest": dest, "send": send, "held": held, "move": move, "offsets": off}


def _alltoallv(ops, x, send_counts, recv_counts, group, backend):
    import torch
    import torch.distributed as dist
    out = ops.empty(int(sum(recv_counts)), backend)
    dist.all_to_all_single(out, ops.to_comm(x, backend), [int(c) for c in recv_counts],
                           [int(c) for c in send_counts], group=group)
    return ops.from_comm(out, backend)


def sharded_sort(keys, group=None, ops=None):
    """Sorts the keys held by all ranks of `group` (this rank's shard:
    `keys`, an int32 tensor holding uint32 words).  Returns (this rank's
    part of the sorted keys, the partition offsets over ranks)."""
    import torch
    import torch.distributed as dist
    backend = dist.get_backend(group)
    P = dist.get_world_size(group)
    me = dist.get_rank(group)
    if ops is None:
        ops = CudaOps(keys.device)
    # 1-2. bucket counts of every rank
    mine = torch.from_numpy(np.asarray(ops.bucket_counts(keys), dtype=np.int64))
    gathered = [torch.zeros(NUM_BUCKETS, dtype=torch.int64) for _ in range(P)]
    if backend == "gloo":
        dist.all_gather(gathered, mine, group=group)
    else:
        dev = [torch.zeros(NUM_BUCKETS, dtype=torch.int64, device=keys.device) for _ in range(P)]
        dist.all_gather(dev, mine.to(keys.device), group=group)
        gathered = [g.cpu() for g in dev]
    counts = torch.stack(gathered).numpy()
    plan = exchange_plan(counts)
    # 3-4. the shard sorted locally is grouped by destination in rank order
    local = ops.sort(keys)
    recv = plan["send"][:, me]
    received = _alltoallv(ops, local, plan["send"][me], recv, group, backend)
    # 5. local sort of the received bucket range
    mine_sorted = ops.sort(received)
    # 6. post-balance to the exact partitions
    out = _alltoallv(ops, mine_sorted, plan["move"][me], plan["move"][:, me], group, backend)
    return out, plan["offsets"]
