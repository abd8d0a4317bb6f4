"""The multi-rank paths on CPU with two gloo ranks.

* Replicas (the benchmark's default): each rank makes its own map; the job
  time is the slowest rank's and the rays add up (weak scaling, no collective
  on the data path).
* One map in strips (paper_2204_10871_gb300.shard): each rank shoots its
  strip of lattice rows and the partial count maps are summed.  The strips
  are shot here by the FP64 oracle (no GPU on this host); the summed map must
  equal the oracle's whole map exactly (integer counts)."""
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


def test_strips_tile_the_lattice():
    from paper_2204_10871_gb300 import shard
    for n in (0, 1, 7, 64, 335, 1000, 20001):
        for world in (1, 2, 3, 8):
            for align in (1, 7, 64, 335):
                strips = [shard.strip_rows(n, world, r, align) for r in range(world)]
                assert strips[0][0] == 0 and strips[-1][1] == n
                assert all(a[1] == b[0] for a, b in zip(strips, strips[1:]))
                assert all(r0 % align == 0 for r0, _ in strips)
                sizes = [(r1 - r0 + align - 1) // align for r0, r1 in strips]
                assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.strip_rows(10, 2, 2)


SHARD_CFG = (0.4, 0.05, 0.3, (-1.5, 1.5, -1.5, 1.5), 24, 9.0)


def _strip_rank(rank, world, port, out):
    import numpy as np
    import oracle
    from paper_2204_10871_gb300 import lensgen, shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    po = oracle.make_params(*SHARD_CFG)
    qo = oracle.size(po)
    xy, m = lensgen.lens_field(30, (qo.a1, qo.a2, qo.b1, qo.b2), seed=3)
    r0, r1 = shard.strip_rows(qo.nry, world, rank, align=5)
    part, _, _ = oracle.make_map(po, qo, xy, m, rows=(r0, r1), threads=1)
    counts = torch.from_numpy(part.copy())
    shard.sum_maps(counts)
    out.put((rank, counts.numpy().tobytes()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_their_strips_into_the_whole_map():
    import numpy as np
    import oracle
    from paper_2204_10871_gb300 import lensgen
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_strip_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    po = oracle.make_params(*SHARD_CFG)
    qo = oracle.size(po)
    xy, m = lensgen.lens_field(30, (qo.a1, qo.a2, qo.b1, qo.b2), seed=3)
    whole, _, _ = oracle.make_map(po, qo, xy, m, threads=1)
    for _, b in res:
        got = np.frombuffer(b, dtype=np.uint32).reshape(whole.shape)
        assert np.array_equal(got, whole)
    assert whole.sum() > 0
