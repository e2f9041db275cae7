"""The benchmark's multi-rank aggregation (replicas, no data-path
collective) on two gloo ranks on the CPU: the step time is the maximum over
ranks and the updates are summed, so `value` is the whole job's rate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        dev = torch.device("cpu")
        t = bench.max_over_ranks(1.0 + r, w, dev)       # step times 1 s and 2 s
        u = bench.sum_over_ranks(10.0 * (r + 1), w, dev)  # 10 and 20 updates
        bench.barrier(w)
        out[r] = (t, u, u / t)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.0, 30.0, 15.0)
