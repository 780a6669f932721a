"""Replicas on several ranks (gloo, CPU): the whole-job throughput is the
summed pixels over the slowest rank's time; each rank's work is its own quad
and no data crosses ranks."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r matched 1000 * (r + 1) pixels in 0.5 * (r + 1) s
    t, v = bench.combine_ranks(0.5 * (rank + 1), 1000 * (rank + 1), world)
    out.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_combine_ranks_gloo(world):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    tmax = 0.5 * world
    px = sum(1000 * (r + 1) for r in range(world))
    for _, t, v in res:
        assert t == pytest.approx(tmax) and v == pytest.approx(px / tmax)


def test_combine_ranks_single():
    import bench
    assert bench.combine_ranks(0.25, 1000, 1) == (0.25, 4000.0)
