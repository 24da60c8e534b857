"""The multi-GPU path is replicas only (one independent problem per rank, no
data-path collective): its host logic with world_size 2 on the gloo backend
(CPU processes): the slowest rank's time, the whole-job throughput, and
dealing the boiling-curve cases out to ranks and gathering them back."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1501_03857_gb300 import replicas as R


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, l = R.rank_env()
        t = R.max_over_ranks(10.0 + 5.0 * rank, dist)
        cases = [("dT", 0.008 + 0.003 * k) for k in range(7)]
        mine = R.shard(cases, r, w)
        results = [(c, r) for c in mine]  # each rank tags what it ran
        full = R.gather_shards(results, r, w, dist)
        q.put((rank, (r, w, l), t, R.job_throughput(w, 1000.0, t), mine, full))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(worker, args=(world, port, q), nprocs=world, join=True, start_method="spawn")
    got = sorted(q.get() for _ in range(world))
    cases = [("dT", 0.008 + 0.003 * k) for k in range(7)]
    for rank, env, t, thr, mine, full in got:
        assert env == (rank, world, rank)
        assert t == 15.0  # the slowest rank's time on both ranks
        assert thr == pytest.approx(2 * 1000.0 / 15e-3)
        assert mine == cases[rank::2]
        assert [c for c, _ in full] == cases  # original order restored
        assert [r for _, r in full] == [k % 2 for k in range(7)]  # who ran what


def test_single_process_is_identity():
    assert R.max_over_ranks(3.5) == 3.5
    assert R.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert R.gather_shards([1, 2, 3], 0, 1) == [1, 2, 3]
    assert R.job_throughput(1, 500.0, 250.0) == 2000.0
