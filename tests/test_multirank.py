"""The benchmark's multi-rank path on CPU (gloo, world size 2): ranks advance
distinct replicas of the workload (weak scaling) and the job time is the slowest
rank's; no collective touches the lattice data.  Each rank runs its own lattice
(through the oracle, on a small extent): mass is conserved on each, the replicas'
random streams differ, and a rank's lattice equals the same replica run alone."""
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
        # each rank's own lattice (the workload's parameters on a small extent): the
        # oracle's state after a few steps, and its mass before and after
        import hashlib
        import oracle as O
        small = dict(cfg, Lx=32, Ly=16)
        ref = O.Lattice(**small)
        s0 = ref.init()
        s = ref.run(s0, 0, 4)
        digest = hashlib.sha256(s.tobytes()).hexdigest()
        gathered = [None] * world
        dist.all_gather_object(gathered, (rank, int(s0.sum()), int(s.sum()), digest))
        q.put((rank, cfg["replica"], slow, gathered))
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
    views = [o[3] for o in out]
    assert views[0] == views[1]                   # both ranks gathered the same records
    (r0, m00, m01, h0), (r1, m10, m11, h1) = views[0]
    assert (r0, r1) == (0, 1)
    assert m00 == m01 and m10 == m11              # mass conserved on every rank
    assert h0 != h1                               # distinct replicas: distinct random streams
    # rank 0's lattice is the replica-0 lattice of one process alone (bit for bit)
    import hashlib
    import bench
    import oracle as O
    from paper_2203_01380_gb300 import inputs
    cfg = dict(bench.rank_workload({k: v for k, v in inputs.LARGE_D2Q5.items() if k != "steps"}, 0), Lx=32, Ly=16)
    ref = O.Lattice(**cfg)
    assert hashlib.sha256(ref.run(ref.init(), 0, 4).tobytes()).hexdigest() == h0


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
