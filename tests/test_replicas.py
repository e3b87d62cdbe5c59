"""The multi-GPU form is replicas: disjoint frame shards per rank, a barrier,
and the slowest rank's time.  Checked on CPU with two gloo ranks."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2304_14492_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://")
    try:
        r, w, local = replicas.dist_env()
        frames = list(replicas.shard(r, 16))
        dist.barrier()
        ms_local = 10.0 + 5.0 * r                      # the ranks finish at different times
        ms = replicas.max_over_ranks(ms_local)
        q.put((r, w, local, frames, ms, replicas.job_throughput(w, 16, 100, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = [set(r[3]) for r in res]
    assert shards[0].isdisjoint(shards[1]) and shards[0] | shards[1] == set(range(32))
    for r, w, local, _, ms, value in res:
        assert w == world and local == r
        assert ms == 15.0                              # the slower rank's time on every rank
        assert value == pytest.approx(world * 16 * 100 / 0.015)


def test_single_process_needs_no_collective():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert list(replicas.shard(0, 4)) == [0, 1, 2, 3]
    assert replicas.job_throughput(1, 16, 10, 2.0) == pytest.approx(80000.0)
