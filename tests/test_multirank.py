"""The replica path of the benchmark for N > 1 ranks, on CPU with two gloo
ranks: the job's time is the slowest rank's, the whole-job rate counts every
rank's units (weak scaling, no exchange on the data path), and each rank
draws its own input shard."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    from paper_1804_10987_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.job_time_ms(10.0 + 5.0 * rank, world, "cpu")
        rate = bench.job_rate(1200, world, t)
        g = torch.Generator()
        g.manual_seed(bench.c4_rank_seed(synth, rank))
        shard = torch.randn(8, generator=g, dtype=torch.float64)
        shards = [torch.zeros(8, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(shards, shard)
        q.put((rank, t, rate, [x.tolist() for x in shards]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_rate_and_shards():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, t, rate, shards in res:
        assert t == 15.0  # the slower rank's time
        assert rate == pytest.approx(2 * 1200 / 0.015)
        assert shards[0] != shards[1]  # distinct input shards
    assert res[0][3] == res[1][3]


def test_single_rank_passes_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(7.5, 1, "cpu") == 7.5
    assert bench.job_rate(9600, 1, 240.0) == pytest.approx(40_000.0)
