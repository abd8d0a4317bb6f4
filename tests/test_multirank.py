"""The benchmark's multi-rank path on CPU: two gloo ranks, each with its own
map time; the job time is the slowest rank's and the rays add up (weak
scaling, no collective on the data path)."""
import os
import socket

import pytest

import bench

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_init() == (world, rank, rank)
    my_ms = 100.0 + 50.0 * rank  # rank 1 is slower
    ms = bench.slowest_rank_ms(my_ms, dist, torch.device("cpu"))
    value = bench.whole_job_rays_per_s(1e9, world, ms / 4)
    out.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    assert all(abs(r[2] - 2 * 1e9 / (150.0 / 4 * 1e-3)) < 1e-3 for r in res)
