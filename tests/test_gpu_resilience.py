"""Checkpoint/resume of the integrator state and the bounded-wait failure path."""
import numpy as np
import pytest

import oracle
from oracle import hermite
from paper_0707_0438_gb300 import abi, workloads
from tests.gpu_util import assert_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_resume_from_checkpoint_is_bitwise_identical(kirin_lib, precision):
    p = workloads.plummer(1024, 1002, eps=1e-3)
    t_mid, t_end = 1.0 / 64, 1.0 / 32
    with abi.Kirin(p.n, p.eps, precision=precision) as k:
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(0.0)
        k.hermite_run(t_end)
        straight = k.get_state()
    with abi.Kirin(p.n, p.eps, precision=precision) as k:
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(0.0)
        k.hermite_run(t_mid)
        ckpt = k.get_state()
    assert ckpt["t"].max() <= t_mid and ckpt["t"].min() < t_mid  # genuinely mid-run for some particles
    with abi.Kirin(p.n, p.eps, precision=precision) as k:  # a fresh context resumes
        k.set_state(p.m, ckpt)
        k.hermite_run(t_end)
        resumed = k.get_state()
    for key in ("x", "v", "a", "j", "t", "dt"):
        assert np.array_equal(resumed[key], straight[key]), key


def test_bounded_wait_times_out_and_context_survives(kirin_lib):
    p = workloads.plummer(500, 4, eps=0.01)
    with abi.Kirin(p.n, p.eps) as k:
        assert k.selftest_wait_timeout(2_000_000) == abi.KIRIN_ETIMEOUT  # 2 ms limit
        k.set_j_particles(p.m, p.x, p.v)
        got = k.forces()
        assert_parity(got, oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps), "mixed")
        k.sync()  # the error flag was cleared when it was reported


def test_arrival_wait_times_out_and_shared_run_continues(kirin_lib):
    """The waits between the CTAs of the single-launch shared steps are bounded: a wait for an
    arrival that never comes gives up (2 ms limit) with KIRIN_ETIMEOUT, and the same context then
    runs shared steps in one launch that match the oracle."""
    p = workloads.plummer(256, 5, eps=1.0 / 256)
    with abi.Kirin(p.n, p.eps, precision="mixed") as k:
        assert k.selftest_arrival_timeout(2_000_000) == abi.KIRIN_ETIMEOUT
        k.set_j_particles(p.m, p.x, p.v)
        assert k.shared_persistent_active()
        k.hermite_init(0.0)
        k.hermite_shared_run(1.0 / 1024, 4)
        st = k.get_state()
    xr, _, _, _, _ = hermite.shared_steps(p.m, p.x, p.v, p.eps, 1.0 / 1024, 4)
    assert np.abs(st["x"] - xr).max() <= 1e-7 * np.abs(p.x).max()


def test_contexts_and_batches_release_device_memory(kirin_lib):
    """Create, use and destroy contexts and batches repeatedly (device-loop graphs, launch tables,
    split partials, the neighbour buffers, batch work lists re-planned): the free device memory
    returns to where it started."""
    import torch
    p = workloads.plummer(20000, 31, eps=1e-3)
    sizes = np.array([300, 1000, 4000])
    cl = [workloads.plummer(int(n), (31, c), eps=1.0 / n) for c, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    bm, bx, bv = (np.concatenate([getattr(c, a) for c in cl]) for a in ("m", "x", "v"))

    def cycle():
        with abi.Kirin(p.n, p.eps) as k:
            k.set_j_particles(p.m, p.x, p.v)
            k.forces(workloads.i_subset(p.n, 100, seed=1))
            k.set_nn(True)
            k.forces(workloads.i_subset(p.n, 37, seed=2))
            k.hermite_init(0.0)
            k.hermite_run(1.0 / 512)
        with abi.KirinBatch(off, [c.eps for c in cl]) as b:
            b.set_state(bm, bx, bv)
            for g, jt in ((2, 2), (4, 1), (1, 0)):
                b.set_launch(g, jt)
                b.accel()
            b.leapfrog(1.0 / 256, 4)
            b.sync()

    cycle()  # first use: lazily loaded modules and the runtime's own pools
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(10):
        cycle()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 <= 8 << 20, (free0 - free1) / 2**20  # MiB lost over ten cycles
