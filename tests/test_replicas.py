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


SUPERHEATS = (0.008, 0.0137, 0.019, 0.025, 0.032)
GWS = (0.0, 0.065)
SEEDS = (1, 2, 3)


def fake_runner(runs, cfg, rv, rl, base, t_switch, t_settle, t_avg, every, stream, log=None):
    """Stands in for the batched GPU run: a deterministic result per
    ((Delta T, G_w), seed) with a flux maximum inside the superheat range."""
    if log is not None:
        log.extend(runs)
    return [{"q_mean": dT * (0.05 - dT) * (1.0 + 0.01 * gw + 0.002 * sd), "q_std": 1e-5 * sd,
             "coverage": [0.1 * (dT > 0.01), 0.3], "bubbles": [2, 5]} for (dT, gw), sd in runs]


def curve(dist=None, log=None):
    from paper_1501_03857_gb300 import experiments as E
    return E.boiling_curve(SUPERHEATS, Gw_values=GWS, seeds=SEEDS, dist=dist,
                           runner=lambda *a: fake_runner(*a, log=log))


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
        ran = []
        c = curve(dist, ran)
        q.put((rank, (r, w, l), t, R.job_throughput(w, 1000.0, t), mine, full, ran, c["cases"], c["curves"]))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(worker, args=(world, port, q), nprocs=world, join=True, start_method="spawn")
    got = sorted((q.get() for _ in range(world)), key=lambda g: g[0])
    cases = [("dT", 0.008 + 0.003 * k) for k in range(7)]
    alone = curve()
    runs = [((float(dT), float(gw)), sd) for gw in GWS for dT in SUPERHEATS for sd in SEEDS]
    for rank, env, t, thr, mine, full, ran, curve_cases, curves in got:
        # a sharded boiling curve: each rank ran every second run, and every
        # rank returns the whole curve, identical to a one-process run
        assert ran == runs[rank::2]
        assert curve_cases == alone["cases"]
        assert curves == alone["curves"]
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
