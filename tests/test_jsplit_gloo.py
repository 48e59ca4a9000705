"""The j partition over several GPUs (the j-split of Sect. 3.2 across ranks), its host-side logic on the
CPU: the parts' j ranges cover the particle set in whole tiles, and the gloo all-gather of
jsplit.TorchAllGather followed by the sum in part order reproduces the FP64 oracle's full sum from the
oracle's partial sums, with world_size 2 (gloo)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_0707_0438_gb300 import abi, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.lib()


@pytest.mark.parametrize("n", [1, 127, 128, 129, 1000, 65536, 100003])
@pytest.mark.parametrize("parts", [1, 2, 3, 8, 1000])
def test_partition_ranges_tile_the_set(lib, n, parts):
    ranges = [abi.j_partition_range(n, r, parts) for r in range(parts)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (b0, e0), (b1, e1) in zip(ranges, ranges[1:]):
        assert e0 == b1  # contiguous and disjoint
    for b, e in ranges:
        assert b <= e and b % 128 == 0 and (e % 128 == 0 or e == n)
    sizes = [-(-(e - b) // 128) for b, e in ranges]  # tiles per part
    assert max(sizes) - min(sizes) <= 1 or n < 128 * parts


def test_partition_rejects_bad_parts(lib):
    for part, parts in ((0, 0), (2, 2), (-1, 2), (0, 4097)):
        with pytest.raises(abi.KirinError):
            abi.j_partition_range(100, part, parts)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_0707_0438_gb300 import abi as kabi
    from paper_0707_0438_gb300 import jsplit, workloads
    p = workloads.plummer(1000, 4321, masses="lognormal", eps=0.01)
    b, e = kabi.j_partition_range(p.n, rank, world)
    m_part = np.zeros_like(p.m)
    m_part[b:e] = p.m[b:e]  # a j outside the part adds exact zeros: the partial sum over [b, e)
    acc, jerk, pot = oracle.acc_jerk_pot(m_part, p.x, p.v, p.eps)
    send = np.concatenate([acc.ravel(), jerk.ravel(), pot])
    recv = np.full(world * send.size, np.nan)
    rc = jsplit.TorchAllGather(device="cpu")(send.ctypes.data, recv.ctypes.data, send.size, None)
    total = np.zeros(send.size)
    for r in range(world):  # part order, as k_sum_parts adds them
        total = total + recv[r * send.size:(r + 1) * send.size]
    q.put((rank, rc, (b, e), recv.tobytes(), total))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_exchange_and_part_order_sum_reproduce_the_oracle(lib):
    import oracle
    from paper_0707_0438_gb300 import workloads
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, rc0, r0, recv0, tot0), (_, rc1, r1, recv1, tot1) = out
    assert rc0 == 0 and rc1 == 0 and r0[1] == r1[0] and r0[0] == 0 and r1[1] == 1000
    assert recv0 == recv1 and np.array_equal(tot0, tot1)  # every rank holds the same bits
    p = workloads.plummer(1000, 4321, masses="lognormal", eps=0.01)
    acc, jerk, pot = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps)
    n = p.n
    got_acc, got_jerk, got_pot = tot0[:3 * n].reshape(n, 3), tot0[3 * n:6 * n].reshape(n, 3), tot0[6 * n:]
    # FP64 sums regrouped into two parts: equal to rounding
    assert np.max(np.linalg.norm(got_acc - acc, axis=1) / np.linalg.norm(acc, axis=1)) < 1e-12
    assert np.max(np.linalg.norm(got_jerk - jerk, axis=1) / np.linalg.norm(jerk, axis=1)) < 1e-12
    assert np.max(np.abs(got_pot - pot) / np.abs(pot)) < 1e-13
