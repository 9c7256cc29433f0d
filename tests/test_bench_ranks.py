"""The benchmark's multi-rank aggregation (replicas on N GPUs) on CPU ranks with
the gloo backend: the timed region is the slowest rank's, and the value counts
every rank's DOF updates."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]
    t = bench.slowest_rank_ms(ms, world, "cpu")
    v = bench.whole_job_value(1000, 10, t, world)
    out[rank] = (t, v)
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        t, v = out[r]
        assert t == 20.0
        assert abs(v - 2 * 1000 * 10 / 0.020) < 1e-6
