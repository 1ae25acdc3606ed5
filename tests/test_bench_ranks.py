"""The host side of bench.py's multi-process run (torchrun, one rank per GPU),
on CPU with the gloo backend and two ranks.  The path shards into independent
replicas (every rank renders its own frames; nothing is exchanged on the data
path), so what the ranks share is the timing: the job takes as long as its
slowest rank, and the whole-job rate is every rank's frames over that time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_s, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        total = bench.job_seconds(local_s[rank], world, "cpu")
        rate, total2 = bench.job_rate(10, local_s[rank], world, "cpu")
        out.put((rank, total, rate, total2))
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_rate_counts_every_rank():
    world, local_s = 2, [0.5, 0.8]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, local_s, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, rate, total2 in res:
        assert total == pytest.approx(0.8) and total2 == pytest.approx(0.8)
        assert rate == pytest.approx(10 * world / 0.8)  # 20 frames over the slowest rank's 0.8 s


def test_one_process_uses_its_own_time():
    import bench
    assert bench.job_seconds(0.25, 1, "cpu") == 0.25
    assert bench.job_rate(5, 0.25, 1, "cpu") == (20.0, 0.25)
