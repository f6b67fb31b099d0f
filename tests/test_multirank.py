"""The benchmark's multi-GPU logic, exercised with world_size-2 gloo ranks on
the CPU: each rank gets its own structures (weak scaling, distinct seeds,
the same work shape), and the whole-job figures sum the updates and take the
slowest rank's time."""
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


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench._workload(64, rank)
    upd, ms = bench.job_totals(1000 * (rank + 1), 10.0 * (rank + 1), world, "cpu")
    q.put((rank, [c.seed for c in w], [c.porosity for c in w], upd, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, e0, u0, m0), (r1, s1, e1, u1, m1) = out
    assert set(s0).isdisjoint(s1)          # different structures per rank
    assert e0 == e1 and len(s0) == len(s1)  # same work shape: weak scaling
    assert u0 == u1 == 3000.0              # updates summed over ranks
    assert m0 == m1 == 20.0                # slowest rank's time


def test_single_rank_totals_are_identity():
    import bench
    assert bench.job_totals(123, 4.5, 1, "cpu") == (123.0, 4.5)
