"""The N > 1 (replica) timing reduction, as world_size-2 gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1112_5588_gb300.replicas import aggregate
    units = 1000.0 * (rank + 1)
    secs = 2.0 if rank == 0 else 5.0
    total, tmax, rate = aggregate(units, secs)
    out.put((rank, total, tmax, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, total, tmax, rate in res:
        assert total == 3000.0 and tmax == 5.0 and rate == pytest.approx(600.0)


def test_aggregate_single_rank_identity():
    from paper_1112_5588_gb300.replicas import aggregate
    assert aggregate(10.0, 4.0) == (10.0, 4.0, 2.5)
