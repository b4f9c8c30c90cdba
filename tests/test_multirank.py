"""Multi-rank (weak-scaling) path of bench.py on CPU: two gloo ranks.  Each rank processes
its own independent signals of the same workload shape; the job's step time is the maximum
over ranks and its throughput counts every rank's samples.  There is no data-path
collective: the only communication is the barrier and this one reduction."""
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


def _worker(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, l = bench.dist_env()
        assert (w, r, l) == (world, rank, rank)
        bench.barrier(world)
        t = bench.max_over_ranks(torch, 1.0 + rank, world)       # rank 1 is the slow one
        wl = bench.BatchWorkload(rank, count=6)
        q.put((rank, t, wl.lengths, float(np.abs(wl.sigs[0]).sum()), wl.samples_per_step()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    (r0, t0, len0, sig0, units0), (r1, t1, len1, sig1, units1) = res
    assert t0 == t1 == 2.0                                       # max over ranks
    assert len0 == len1 and units0 == units1                     # same per-rank work (weak scaling)
    assert sig0 != sig1                                          # independent signals per rank
    import bench
    assert bench.job_throughput(world, units0, 2.0) == 2 * units0 / 2.0
