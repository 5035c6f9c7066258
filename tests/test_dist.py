"""The multi-GPU path of bench.py is replicas only (one independent solve per
rank, no data-path collective); its host logic — the barrier and the maximum
of the timed region over ranks, and the whole-job value — is exercised here
with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as tdist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    tdist.barrier()
    local = 1.5 + rank          # rank 1 is the slow one
    tmax = bench.max_over_ranks(local, tdist, torch.device("cpu"))
    value = bench.replica_value(tmax, steps=4, world_size=world)
    out.put((rank, tmax, value, bench.dist_env()))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_rank_timing_reduction():
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
    for rank, tmax, value, env in res:
        assert tmax == 2.5                       # the slowest rank's time, on every rank
        assert value == pytest.approx(2.5 / 8)   # 8 solves over the job
        assert env == (2, rank, 0)
