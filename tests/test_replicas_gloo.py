"""Replica scaling (no data-path collective): two gloo ranks on the CPU run the bench's
whole-job aggregation (slowest rank's time, products of all ranks) and its seeding."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank            # rank 1 is the slowest
        products = 1e6 * (rank + 1)
        out[rank] = (bench.reduce_over_ranks(ms, products, world, "cpu"), bench.replica_seed("plain_large", rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    (ms0, prod0), seed0 = res[0]
    (ms1, prod1), seed1 = res[1]
    assert ms0 == ms1 == 15.0                 # max over ranks
    assert prod0 == prod1 == 3e6              # sum over ranks
    assert seed0 != seed1                     # independent replicas


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(7.0, 5.0, 1, "cpu") == (7.0, 5.0)
