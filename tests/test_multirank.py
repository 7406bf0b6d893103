"""The multi-GPU path of the benchmark on CPU: two gloo ranks (world size 2).

Worlds are independent, so ranks shard them with no data-path collective:
each rank builds its own worlds (disjoint seeds), and the job's CASPS is the
agents all ranks stepped over the slowest rank's time.  This runs the same
host-side code as bench.py under torchrun, with gloo on the CPU instead of
NCCL on GPUs.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        sc = bench.make_scene("256x16", rank)
        first_x = float(sc.px[0])
        # rank r "stepped" 100 + r agents for 10 steps in 1 + r seconds
        casps, e2e = bench.combine_over_ranks(1.0 + rank, 2.0 + rank, 100 + rank, 10, 5, dist, torch, "cpu")
        dist.barrier()
        out.put((rank, sc.num_worlds, sc.num_agents, first_x, casps, e2e))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_worlds_and_combine_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, a0, x0, c0, e0), (r1, w1, a1, x1, c1, e1) = res
    assert (w0, a0) == (w1, a1) == (256, 4096)          # weak scaling: the same work per rank
    assert x0 != x1                                       # but different worlds (disjoint seeds)
    expect = (100 + 101) * 10 / 2.0                       # agents summed, the slowest rank's time
    assert c0 == c1 == pytest.approx(expect)
    assert e0 == e1 == pytest.approx((100 + 101) * 5 / 3.0)


def test_single_rank_needs_no_collective():
    import bench
    casps, e2e = bench.combine_over_ranks(2.0, 4.0, 50, 10, 6, None, torch, "cpu")
    assert casps == pytest.approx(250.0) and e2e == pytest.approx(75.0)
