"""The multi-rank logic of bench.py on CPU with the gloo backend (world size
2): every rank computes its own copy of the workload (independent problems,
no collective on the data path); the reported value is the units of all
ranks over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    ms = 10.0 * (rank + 1)          # rank 1 is the slower one
    slow = bench.max_over_ranks(ms, dist, "cpu")
    out.put((rank, slow, bench.whole_job_rate(2, world, slow)))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_max_over_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(world))
    assert [r[1] for r in res] == [20.0, 20.0]
    assert [r[2] for r in res] == [200.0, 200.0]   # 2 dets x 2 ranks / 20 ms


def test_bench_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.whole_job_rate(2, 1, 500.0) == 4.0
