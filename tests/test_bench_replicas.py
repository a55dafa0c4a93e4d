"""The multi-GPU form is replicas (every rank sorts its own 2^26 keys, no
collective on the data path).  bench.py's only cross-rank step is taking the
slowest rank's time; check it with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is slower
    job = bench.max_over_ranks(ms, world, torch.device("cpu"))
    out[rank] = (job, bench.whole_job_rate(1 << 26, world, 4, job))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    job, rate = res[0]
    assert job == 15.0
    assert rate == pytest.approx(2 * (1 << 26) * 4 / 0.015 / 1e9)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.whole_job_rate(100, 1, 2, 1.0) == pytest.approx(200 / 1e-3 / 1e9)
