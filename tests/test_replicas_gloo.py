"""The multi-GPU path is replicas only: each rank runs its own solve and the
only collectives are the barrier and the max (or min) over ranks of timed
quantities.  That host-side logic runs here on CPU with two gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [12.5, 30.25][rank]
    local_rate = [4.0e9, 3.0e9][rank]
    dist.barrier()
    out[rank] = (bench.max_over_ranks(local_ms), bench.max_over_ranks(local_rate, op="min"))
    dist.destroy_process_group()


def test_two_rank_max_and_min_over_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (30.25, 3.0e9)


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(7.0) == 7.0
