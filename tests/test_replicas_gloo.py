"""Multi-GPU is replicas only: N ranks transpose their own graphs with no
collective on the data path; the bench takes the max step time over ranks.
This covers that host logic with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [10.0, 12.5][rank]
    ms, value = bench.aggregate_ranks(ms_local, 1000, world)
    out[rank] = (ms, value, bench.replica_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, value, _ = out[r]
        assert ms == 12.5
        assert value == pytest.approx(2 * 1000 / 12.5e-3)
    assert out[0][2] != out[1][2]


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.aggregate_ranks(4.0, 1000, 1)
    assert ms == 4.0 and value == pytest.approx(1000 / 4e-3)
