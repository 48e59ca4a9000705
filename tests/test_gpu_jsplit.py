"""The j partition across GPUs (the j-split of Sect. 3.2 lifted to ranks), on one GPU: contexts that
each sum one part of the j tiles give partial sums that add up to the oracle's forces, and contexts
driven by host threads that exchange through jsplit.LocalAllGather integrate block steps in lockstep,
every part holding the same bits, as an unpartitioned context does."""
import threading

import numpy as np
import pytest

import oracle
from paper_0707_0438_gb300 import abi, jsplit, metrics, workloads
from tests.gpu_util import assert_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("n,parts,n_i", [(5000, 2, None), (5000, 3, 700), (300, 4, None), (40000, 2, 5)])
def test_parts_add_up_to_the_oracle(kirin_lib, precision, n, parts, n_i):
    """Each part's partial sums; their sum over the parts against the oracle's full sum (a ragged set,
    more parts than tiles (300 j are 3 tiles: one part sums nothing), and a tiny block)."""
    p = workloads.plummer(n, (77, n), masses="lognormal", eps=1.0 / 256)
    il = None if n_i is None else workloads.i_subset(n, n_i, seed=4)
    tot = None
    for r in range(parts):
        with abi.Kirin(n, p.eps, precision=precision) as k:
            k.set_j_particles(p.m, p.x, p.v)
            k.set_j_partition(r, parts)
            got = k.forces(il)
        b, e = abi.j_partition_range(n, r, parts)
        if b == e:
            assert all(np.all(q == 0.0) for q in got)
        if precision == "fp64" and b < e:
            m_part = np.zeros_like(p.m)
            m_part[b:e] = p.m[b:e]
            ref_part = oracle.acc_jerk_pot(m_part, p.x, p.v, p.eps, i_idx=il)
            assert np.max(metrics.rel_err_vec(got[0], ref_part[0])) < 1e-10
        tot = got if tot is None else tuple(a + g for a, g in zip(tot, got))
    assert_parity(tot, oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il), precision, f"{parts} parts")


def _run_parts(p, parts, precision, t_end, eps):
    """Block-step Hermite runs of `parts` partitioned contexts on GPU 0, one host thread each."""
    ex = jsplit.LocalAllGather([0] * parts)
    out = [None] * parts
    errs = []

    def drive(r):
        try:
            with abi.Kirin(p.n, eps, precision=precision) as k:
                k.set_j_particles(p.m, p.x, p.v)
                k.set_j_partition(r, parts, ex.for_part(r))
                e0 = sum(k.energy())
                full = k.forces()  # whole sums through the exchange
                k.hermite_init(0.0)
                steps, _ = k.hermite_run(t_end)  # a partitioned context steps from the host
                out[r] = (full, steps, k.get_state(), e0, sum(k.energy()))
        except BaseException as exc:  # surfaced below; the barrier times out for the others
            errs.append(exc)
            ex.barrier.abort()

    th = [threading.Thread(target=drive, args=(r,)) for r in range(parts)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_threaded_parts_integrate_block_steps_in_lockstep(kirin_lib, precision):
    p = workloads.plummer(2048, 2222, eps=0.01)
    t_end = 1.0 / 64
    out = _run_parts(p, 2, precision, t_end, p.eps)
    (f0, s0, st0, e00, e10), (f1, s1, st1, _, _) = out
    # every part holds the same bits: forces, schedule and final state
    assert s0 == s1 and s0 > 20
    for a, b in zip(f0, f1):
        assert np.array_equal(a, b)
    for q in ("x", "v", "a", "j", "t", "dt"):
        assert np.array_equal(st0[q], st1[q]), q
    assert_parity(f0, oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps), precision, "exchanged forces")
    assert abs(metrics.energy_error(e00, e10)) < 1e-6
    # against one unpartitioned context on the same run
    with abi.Kirin(p.n, p.eps, precision=precision) as k:
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(0.0)
        steps, _ = k.hermite_run(t_end)
        ref = k.get_state()
    if precision == "fp64":  # the same schedule; positions equal to the rounding of regrouped sums
        assert steps == s0 and np.array_equal(ref["t"], st0["t"]) and np.array_equal(ref["dt"], st0["dt"])
        assert np.abs(ref["x"] - st0["x"]).max() <= 1e-12 * np.abs(p.x).max()
    else:
        assert abs(steps - s0) <= 2
        assert np.abs(ref["x"] - st0["x"]).max() <= 1e-6 * np.abs(p.x).max()


def test_exchange_failures_are_reported(kirin_lib):
    p = workloads.plummer(600, 5, eps=0.01)
    with abi.Kirin(p.n, p.eps, precision="mixed") as k:
        k.set_j_particles(p.m, p.x, p.v)
        k.set_j_partition(0, 2, lambda send, recv, count, stream: 3)
        with pytest.raises(abi.KirinError) as ei:
            k.forces()
        assert ei.value.code == abi.KIRIN_EEXCHANGE

        def broken(send, recv, count, stream):
            raise ValueError("peer went away")
        k.set_j_partition(1, 2, broken)
        with pytest.raises(abi.KirinError) as ei:
            k.forces()
        assert ei.value.code == abi.KIRIN_EEXCHANGE and isinstance(ei.value.__cause__, ValueError)
        # calls without a j-partition form refuse; n_parts = 1 restores the whole sum
        import torch
        dev = torch.device("cuda:0")
        m, x = torch.tensor(p.m, device=dev), torch.tensor(p.x, device=dev)
        gx, gm = torch.empty_like(x), torch.empty_like(m)
        with pytest.raises(abi.KirinError) as ei:
            k.accel_adjoint_dev(m, x, x, gx, gm)
        assert ei.value.code == abi.KIRIN_ESTATE
        k.set_j_partition(0, 1)
        got = k.forces()
    assert_parity(got, oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps), "mixed")


def test_torch_allgather_on_device_buffers_over_nccl(kirin_lib):
    """jsplit.TorchAllGather on CUDA device pointers, as kirin_set_j_partition calls it, over an NCCL
    group of one rank (this runs on one GPU): the device views, the stream ordering against the
    context's stream and the gathered layout."""
    import os
    import socket

    import torch
    import torch.distributed as dist
    dev = torch.device("cuda:0")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=dev)
    try:
        side = torch.cuda.Stream(device=dev)
        send = torch.empty(7 * 37, dtype=torch.float64, device=dev)
        recv = torch.full((7 * 37,), float("nan"), dtype=torch.float64, device=dev)
        with torch.cuda.stream(side):
            send.copy_(torch.arange(7 * 37, dtype=torch.float64, device=dev))  # enqueued before the call
        rc = jsplit.TorchAllGather(device=dev)(send.data_ptr(), recv.data_ptr(), send.numel(), side.cuda_stream)
        side.synchronize()
        assert rc == 0 and torch.equal(recv, send)
        # and through a context: with one part the callback is never needed, the sums are whole
        p = workloads.plummer(700, 41, eps=0.01)
        with abi.Kirin(p.n, p.eps, precision="fp64") as k:
            k.set_j_particles(p.m, p.x, p.v)
            k.set_j_partition(0, 1, jsplit.TorchAllGather(device=dev))
            got = k.forces()
        assert_parity(got, oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps), "fp64")
    finally:
        dist.destroy_process_group()


def test_threaded_parts_leapfrog_in_lockstep(kirin_lib):
    """The force-only calls of the leapfrog (Sect. 4.3 client) through the exchange: two threaded parts
    give the same bits, and the unpartitioned context's trajectory to rounding (FP64)."""
    import torch
    dev = torch.device("cuda:0")
    p = workloads.plummer(3000, 4444, eps=0.02)
    ex = jsplit.LocalAllGather([0, 0])
    out, errs = [None, None], []

    def drive(r):
        try:
            with abi.Kirin(p.n, p.eps, precision="fp64") as k:
                k.set_j_partition(r, 2, ex.for_part(r))
                m, x, v = (torch.tensor(a, device=dev) for a in (p.m, p.x, p.v))
                acc = torch.empty_like(x)
                k.leapfrog_dev(m, x, v, acc, 1.0 / 128, 8)
                k.sync()
                out[r] = (x.cpu().numpy(), v.cpu().numpy())
        except BaseException as exc:
            errs.append(exc)
            ex.barrier.abort()

    th = [threading.Thread(target=drive, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    with abi.Kirin(p.n, p.eps, precision="fp64") as k:
        m, x, v = (torch.tensor(a, device=dev) for a in (p.m, p.x, p.v))
        acc = torch.empty_like(x)
        k.leapfrog_dev(m, x, v, acc, 1.0 / 128, 8)
        k.sync()
        ref = x.cpu().numpy()
    assert np.abs(out[0][0] - ref).max() <= 1e-12 * np.abs(p.x).max()
