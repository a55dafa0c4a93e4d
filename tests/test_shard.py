"""The sort across ranks (the paper's machine-level algorithm, Sec. 3):
its exchange plan on the host, and two gloo ranks on CPU whose rank-local
steps (bucket counts, sorting) are done here with numpy, checked against
the oracle's sort of all the keys split into the equal partitions."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_cs_0004013_gb300 import shard


class NumpyOps:
    """Rank-local steps on the host (test infrastructure: the product's
    rank-local steps are librsort's kernels, CudaOps)."""

    def bucket_counts(self, keys):
        w = keys.numpy().view(np.uint32)
        return np.bincount(w >> np.uint32(shard.BUCKET_SHIFT), minlength=shard.NUM_BUCKETS).astype(np.int64)

    def sort(self, keys):
        import torch
        return torch.from_numpy(oracle.sort_keys(keys.numpy().view(np.uint32)).view(np.int32).copy())

    def to_comm(self, x, backend):
        return x

    def from_comm(self, x, backend):
        return x

    def empty(self, n, backend):
        import torch
        return torch.empty(n, dtype=torch.int32)


def test_partition_offsets_match_the_oracle():
    for total, parts in ((0, 3), (10, 3), (64, 64), (1000, 7)):
        assert np.array_equal(shard.partition_offsets_of(total, parts), oracle.partition_offsets(total, parts))


def test_exchange_plan_by_hand():
    """Two ranks, four buckets: counts [[3, 0, 1, 2], [1, 2, 0, 3]] -> totals
    [4, 2, 1, 5] (12 keys), partitions [0, 6) and [6, 12).  Bucket starts 0,
    4, 6, 7 -> ranks 0, 0, 1, 1.  Rank 0 sends 3 to itself and 3 to rank 1;
    rank 1 sends 3 and 3.  Each holds 6: already its partition."""
    c = np.zeros((2, shard.NUM_BUCKETS), np.int64)
    c[0, :4] = [3, 0, 1, 2]
    c[1, :4] = [1, 2, 0, 3]
    p = shard.exchange_plan(c)
    assert list(p["dest"][:4]) == [0, 0, 1, 1]
    assert p["send"].tolist() == [[3, 3], [3, 3]]
    assert p["held"].tolist() == [6, 6]
    assert p["move"].tolist() == [[6, 0], [0, 6]]


def test_exchange_plan_post_balance():
    """One big bucket holds most keys: it goes to one rank whole, and the
    post-balance spreads it over the exact partitions."""
    rng = np.random.default_rng(1)
    for P in (2, 3, 5):
        c = rng.integers(0, 50, (P, shard.NUM_BUCKETS)).astype(np.int64)
        c[:, 7] += 10000
        p = shard.exchange_plan(c)
        total = int(c.sum())
        assert p["send"].sum() == total and p["held"].sum() == total
        assert np.array_equal(p["send"].sum(axis=1), c.sum(axis=1))  # every rank sends all its keys
        assert np.array_equal(p["move"].sum(axis=1), p["held"])  # and then everything it holds
        assert np.array_equal(p["move"].sum(axis=0), np.diff(p["offsets"]))  # into the exact partitions
        assert np.all(np.diff(p["dest"]) >= 0)  # contiguous bucket ranges per rank


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, shards, out_dir, use_cuda):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        keys = shards[rank]
        if use_cuda:
            t = torch.from_numpy(keys.view(np.int32).copy()).cuda()
            out, offs = shard.sharded_sort(t, ops=shard.CudaOps("cuda:0"))
            out = out.cpu()
        else:
            t = torch.from_numpy(keys.view(np.int32).copy())
            out, offs = shard.sharded_sort(t, ops=NumpyOps())
        np.save(os.path.join(out_dir, f"r{rank}.npy"), out.numpy().view(np.uint32))
        np.save(os.path.join(out_dir, "offs.npy"), offs)
    finally:
        dist.destroy_process_group()


def run_ranks(shards, tmp_path, use_cuda=False):
    import torch.multiprocessing as mp
    world = len(shards)
    mp.spawn(_rank_main, args=(world, _free_port(), shards, str(tmp_path), use_cuda), nprocs=world, join=True)
    allk = np.concatenate(shards)
    want = oracle.sort_keys(allk)
    offs = oracle.partition_offsets(allk.size, world)
    assert np.array_equal(np.load(tmp_path / "offs.npy"), offs)
    for r in range(world):
        got = np.load(tmp_path / f"r{r}.npy")
        assert np.array_equal(got, want[int(offs[r]): int(offs[r + 1])]), r


@pytest.mark.parametrize("case", ["uneven", "clustered", "one_empty"])
def test_two_gloo_ranks(tmp_path, case):
    if case == "uneven":
        shards = [synth.uniform31(30001, 1), synth.uniform31(7777, 2)]
    elif case == "clustered":  # most keys in one bucket: the post-balance moves them
        shards = [synth.tight_clusters(20000, 3), synth.few_distinct(15000, 4)]
    else:
        shards = [np.zeros(0, np.uint32), synth.uniform31(5000, 5) | (synth.uniform31(5000, 6) << np.uint32(1))]
    run_ranks(shards, tmp_path)


def test_three_gloo_ranks(tmp_path):
    run_ranks([synth.gauss_mix(12000, 7), synth.uniform31(1, 8), synth.skewed_chunks(9000, 9)], tmp_path)
