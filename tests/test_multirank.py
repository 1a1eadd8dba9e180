"""The benchmark's multi-rank path on CPU (gloo, world size 2): ranks advance
distinct replicas of the workload (weak scaling) and the job time is the slowest
rank's; no collective touches the lattice data."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import bench
    from paper_2203_01380_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg = bench.rank_workload({k: v for k, v in inputs.LARGE_D2Q5.items() if k != "steps"}, rank)
        slow = bench.max_over_ranks(10.0 * (rank + 1), world)
        q.put((rank, cfg["replica"], slow))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [0, 1]          # one replica per rank
    assert all(o[2] == 20.0 for o in out)         # every rank sees the slowest time


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
