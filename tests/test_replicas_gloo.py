"""Multi-GPU runs are replicas (each rank evaluates its own copy of the workload, no
data-path collective): the whole-job rate is all ranks' work over the slowest rank's
time.  Checked with world_size 2 on the CPU (gloo)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank 1 is the slow one
    rate, t_max = bench.replica_rate(2.0 + rank, units_per_step=1e12, steps=4, world=world, dist=dist,
                                     device="cpu")
    q.put((rank, rate, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_rate_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, t_max in out:
        assert t_max == pytest.approx(3.0)
        assert rate == pytest.approx(2 * 1e12 * 4 / 3.0)


def test_single_rank_needs_no_collective():
    import bench
    rate, t = bench.replica_rate(2.0, 1e12, 4, 1)
    assert t == 2.0 and rate == pytest.approx(2e12)
