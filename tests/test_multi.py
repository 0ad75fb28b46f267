"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every
rank runs the whole workload (replicas, weak scaling), the timed region is
bracketed by barriers, the time is the maximum over ranks and the whole-job
rate counts the units of all ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    local_s = 1.0 + rank                   # rank 1 is the slow one
    t = bench.reduce_max(local_s, w)
    out[rank] = (t, bench.whole_job_value(256, w, t / 10))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, v = out[r]
        assert t == pytest.approx(2.0)                 # max over ranks
        assert v == pytest.approx(256 * 2 / 0.2)       # all ranks' products / slowest time per step
