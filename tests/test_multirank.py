"""Multi-rank host logic of bench.py on CPU: two gloo ranks on 127.0.0.1.

A multi-GPU run is N independent replicas (one box per rank, seed + rank, no
data-path collective); ranks meet only for the barrier and the max-over-ranks
time, and the whole-job throughput counts the cells of every rank over the
slowest rank's time.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        t_local = 1.0 + 0.5 * rank  # rank 1 is the slow one
        t = bench.max_over_ranks(t_local, world, device="cpu")
        dist.barrier()
        cfg = dict(N=32, nu=0.005, tau_p=[0.05], Y0=[0.01], mach_rms=0.2, k0=4.0, seed=7)
        box = bench.rank_box(cfg, rank)
        rate = bench.job_rate(32.0 ** 3, 10, world, t)
        with open(os.path.join(outdir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r %r" % (t, box["seed"], rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.spawn(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    got = [open(tmp_path / ("rank%d.txt" % r)).read().split() for r in range(world)]
    times = [float(g[0]) for g in got]
    seeds = [int(g[1]) for g in got]
    rates = [float(g[2]) for g in got]
    assert times == [1.5, 1.5]                      # every rank sees the slowest rank's time
    assert seeds == [7, 8]                          # independent replicas: seed + rank
    assert rates[0] == rates[1] == pytest.approx(32.0 ** 3 * 10 * 2 / 1.5)  # all ranks' cells / max time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_rate(100.0, 4, 1, 2.0) == 200.0
