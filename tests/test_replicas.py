"""Multi-process host logic of the replica runs (world size 2, gloo, CPU): every rank sees the
slowest rank's time, and the job's seconds per timestep count every rank's timesteps."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2411_14847_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 * (rank + 1)                      # rank 1 is the slow one
        dist.barrier()
        m = replicas.max_over_ranks(ms, dist)
        q.put((rank, m, replicas.seconds_per_timestep(m, 3, world), replicas.replica_seed(1003, rank)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, PORT, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[1] for r in res] == [200.0, 200.0]
    assert res[0][2] == pytest.approx(200.0 / 1e3 / 6)
    assert res[0][3] != res[1][3]


PORT = _free_port()


def test_single_process_is_identity():
    assert replicas.max_over_ranks(12.5) == 12.5
    assert replicas.seconds_per_timestep(1500.0, 3, 1) == pytest.approx(0.5)
