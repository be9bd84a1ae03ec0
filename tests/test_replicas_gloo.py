"""Host logic of multi-GPU runs (independent replicas, no collective on the
data path): the timing reduction over ranks and the whole-job throughput,
run as world_size-2 gloo process groups on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        worst = bench.max_over_ranks(times[rank], dist, "cpu")
        dist.barrier()
        out[rank] = (worst, bench.replica_throughput(1000, world, worst))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(0.010, 0.012), (0.5, 0.25)])
def test_max_over_ranks_and_throughput(times):
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    worst = max(times)
    for r in range(world):
        assert out[r][0] == pytest.approx(worst)
        assert out[r][1] == pytest.approx(world * 1000 / worst)


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(0.25) == 0.25
    assert bench.replica_throughput(10, 1, 0.5) == 20.0
