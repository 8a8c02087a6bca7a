"""Replica bookkeeping over ranks, run as two gloo processes on the CPU."""
import os
import socket

import pytest

from paper_2602_14016_gb300 import replicas


@pytest.mark.parametrize("count,world", [(7, 2), (7, 3), (256, 8), (3, 4), (0, 2)])
def test_shards_cover_every_member_once(count, world):
    seen = []
    for r in range(world):
        a, b = replicas.shard(count, r, world)
        assert 0 <= a <= b <= count
        seen.extend(range(a, b))
    assert sorted(seen) == list(range(count))
    sizes = [replicas.shard(count, r, world)[1] - replicas.shard(count, r, world)[0] for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b = replicas.shard(7, rank, world)
        seconds = 1.0 + rank  # the slower rank sets the time
        rate = replicas.whole_job_rate(units_per_rank=(b - a) * 100.0, seconds_per_rank=seconds)
        q.put((rank, replicas.max_over_ranks(seconds), replicas.sum_over_ranks(b - a), rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_units():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, tmax, members, rate in got:
        assert tmax == 2.0
        assert members == 7
        assert abs(rate - 700.0 / 2.0) < 1e-12
