"""GPU parity of the integrator glue (Hermite shared and block steps, energy),
the acceleration/adjoint entry points and the batched ensemble, against the oracle."""
import numpy as np
import pytest

import oracle
from oracle import hermite, leapfrog
from paper_0707_0438_gb300 import abi, metrics, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-7)])
def test_hermite_shared_steps_small_config(kirin_lib, precision, tol):
    """N = 1024, eps = 1/256: one full evaluation and 10 shared Hermite steps, dt = 1/1024."""
    p = workloads.config_small()
    dt, steps = 1.0 / 1024, 10
    xr, vr, ar, jr, _ = hermite.shared_steps(p.m, p.x, p.v, p.eps, dt, steps)
    with abi.Kirin(p.n, p.eps, precision=precision) as k:
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(0.0)
        for _ in range(steps):
            k.hermite_shared_step(dt)
        st = k.get_state()
    scale_x = np.abs(p.x).max()
    assert np.abs(st["x"] - xr).max() <= tol * scale_x
    assert np.abs(st["v"] - vr).max() <= tol * 10 * np.abs(p.v).max()
    assert np.median(metrics.rel_err_vec(st["a"], ar)) <= (1e-12 if precision == "fp64" else 1e-6)
    assert np.all(st["t"] == steps * dt)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shared_run_is_repeated_shared_steps(kirin_lib, precision):
    """kirin_hermite_shared_run(dt, 10) enqueues the same kernels as 10 single steps: identical state."""
    p = workloads.config_small()
    out = []
    for run in (True, False):
        with abi.Kirin(p.n, p.eps, precision=precision) as k:
            k.set_j_particles(p.m, p.x, p.v)
            k.hermite_init(0.0)
            if run:
                k.hermite_shared_run(1.0 / 1024, 10)
            else:
                for _ in range(10):
                    k.hermite_shared_step(1.0 / 1024)
            out.append(k.get_state())
    for key in ("x", "v", "a", "j", "t", "dt"):
        assert np.array_equal(out[0][key], out[1][key]), key
    assert np.all(out[0]["t"] == 10.0 / 1024)


def test_hermite_block_steps_fp64_follow_the_oracle(kirin_lib):
    """Block time-steps (Aarseth criterion, power-of-two levels): same schedule and state as the oracle."""
    p = workloads.plummer(256, 1002, eps=1e-3)
    t_end = 1.0 / 8  # a multiple of the largest step, so every particle ends there
    ref = hermite.block_steps(p.m, p.x, p.v, p.eps, t_end=t_end)
    with abi.Kirin(p.n, p.eps, precision="fp64") as k:
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(0.0)
        blocks = []
        while True:
            t, n_act = k.hermite_block_step(t_end)
            if n_act == 0:
                break
            blocks.append(n_act)
        st = k.get_state()
        kin, pot = k.energy()
    assert blocks == ref["blocks"]
    assert np.array_equal(st["t"], ref["t"]) and np.all(st["t"] == t_end)
    assert np.array_equal(st["dt"], ref["dt"])
    assert np.abs(st["x"] - ref["x"]).max() <= 1e-9
    e_end = kin + pot
    assert e_end == pytest.approx(ref["e_end"], rel=1e-10)


def test_hermite_block_run_energy_drift_mixed_vs_fp64(kirin_lib):
    p = workloads.plummer(2048, 1002, eps=1e-3)
    out = {}
    for precision in ("fp64", "mixed"):
        with abi.Kirin(p.n, p.eps, precision=precision) as k:
            k.set_j_particles(p.m, p.x, p.v)
            e0 = sum(k.energy())
            k.hermite_init(0.0)
            steps, pairs = k.hermite_run(1.0 / 64)
            e1 = sum(k.energy())
            out[precision] = metrics.energy_error(e0, e1)
            assert steps > 0 and pairs > 0
    assert abs(out["fp64"]) < 1e-6
    assert abs(out["mixed"]) < 1e-5


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-7), ("fp64", 1e-11)])
def test_device_leapfrog_is_time_reversible(kirin_lib, precision, tol):
    """kirin_leapfrog_dev at N = 16384: 32 steps forward, velocities negated, 32 steps forward again
    return the initial positions and velocities; the mixed forces differ only by rounding between the
    two passes, the FP64 ones hardly at all."""
    import torch
    dev = torch.device("cuda:0")
    p = workloads.config_adjoint(16384)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    with abi.Kirin(p.n, p.eps, precision=precision, stream=torch.cuda.current_stream().cuda_stream) as k:
        m, x, v = T(p.m), T(p.x), T(p.v)
        acc = torch.empty_like(x)
        k.leapfrog_dev(m, x, v, acc, 1.0 / 128, 32)
        moved = float((x - T(p.x)).abs().max())
        v.neg_()
        k.leapfrog_dev(m, x, v, acc, 1.0 / 128, 32, acc_valid=True)
        k.sync()
        dx = float((x - T(p.x)).abs().max())
        dv = float((-v - T(p.v)).abs().max())
    assert moved > 1e-3
    assert dx <= tol * np.abs(p.x).max() and dv <= tol * 10 * np.abs(p.v).max(), (dx, dv)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_accel_and_adjoint_dev(kirin_lib, precision):
    import torch
    p = workloads.plummer(3000, 1005, eps=0.01)
    dev = torch.device("cuda:0")
    m = torch.tensor(p.m, device=dev)
    x = torch.tensor(p.x, device=dev)
    g = torch.tensor(np.random.default_rng(1).standard_normal((p.n, 3)), device=dev)
    acc = torch.empty_like(x)
    pot = torch.empty_like(m)
    gx = torch.empty_like(x)
    gm = torch.empty_like(m)
    with abi.Kirin(p.n, p.eps, precision=precision, stream=torch.cuda.current_stream().cuda_stream) as k:
        k.accel_dev(m, x, acc, pot)
        k.accel_adjoint_dev(m, x, g, gx, gm)
        k.sync()
    ra, rp = oracle.acc_pot(p.m, p.x, p.eps)
    rgx, rgm = oracle.force_adjoint(p.m, p.x, g.cpu().numpy(), p.eps)
    if precision == "fp64":
        tol_med, tol_max = 1e-12, 1e-10
    else:
        tol_med, tol_max = 1e-6, 1e-5
    e = metrics.rel_err_vec(acc.cpu().numpy(), ra)
    assert np.median(e) <= tol_med and e.max() <= tol_max, ("acc", np.median(e), e.max())
    e = metrics.rel_err_scalar(pot.cpu().numpy(), rp)
    assert np.median(e) <= tol_med and e.max() <= tol_max, ("pot", np.median(e), e.max())
    # The adjoint sums are random-sign sums over j (g is random), and some particles' sums
    # nearly cancel: the per-particle median is held to the force tolerance and the worst
    # particle's error is measured against the RMS size of the gradient.
    for name, got, ref in (("dL/dx", gx.cpu().numpy(), rgx), ("dL/dm", gm.cpu().numpy()[:, None], rgm[:, None])):
        err = np.linalg.norm(got - ref, axis=1)
        rms = np.sqrt(np.mean(np.sum(ref * ref, axis=1)))
        med = np.median(err / np.linalg.norm(ref, axis=1))
        assert med <= tol_med and err.max() / rms <= tol_max, (name, med, err.max() / rms)


def _small_ensemble(n_clusters=24, seed=77):
    return workloads.ensemble(n_clusters, seed=seed, n_lo=64, ratio=40.0)


def test_batched_accelerations_match_per_cluster_oracle(kirin_lib):
    clusters, sizes = _small_ensemble()
    off = np.concatenate([[0], np.cumsum(sizes)])
    m = np.concatenate([c.m for c in clusters])
    x = np.concatenate([c.x for c in clusters])
    v = np.concatenate([c.v for c in clusters])
    b = abi.KirinBatch(off, [c.eps for c in clusters])
    b.set_state(m, x, v)
    acc = b.accel()
    b.close()
    for c, cl in enumerate(clusters):
        ra, _ = oracle.acc_pot(cl.m, cl.x, cl.eps)
        e = metrics.rel_err_vec(acc[off[c]:off[c + 1]], ra)
        assert np.median(e) <= 1e-6 and e.max() <= 1e-5, (c, np.median(e), e.max())


def test_batched_leapfrog_matches_oracle_and_graph_is_identical(kirin_lib):
    clusters, sizes = _small_ensemble(12, seed=5)
    off = np.concatenate([[0], np.cumsum(sizes)])
    m = np.concatenate([c.m for c in clusters])
    x = np.concatenate([c.x for c in clusters])
    v = np.concatenate([c.v for c in clusters])
    dt, steps = 1.0 / 256, 8
    finals = []
    for use_graph in (False, True):
        b = abi.KirinBatch(off, [c.eps for c in clusters])
        b.set_state(m, x, v)
        b.leapfrog(dt, steps, use_graph=use_graph)
        b.sync()
        finals.append(b.get_state())
        b.close()
    assert np.array_equal(finals[0][0], finals[1][0]) and np.array_equal(finals[0][1], finals[1][1])
    xg = finals[1][0]
    for c, cl in enumerate(clusters):
        xs, _ = leapfrog.trajectory(cl.m, cl.x, cl.v, cl.eps, dt, steps)
        # an acceleration error da moves positions by at most ~ (steps dt)^2 / 2 * da over the
        # trajectory; the mixed forces are within 1e-5 |a| per particle
        a0, _ = oracle.acc_pot(cl.m, cl.x, cl.eps)
        bound = 10 * 0.5 * (steps * dt) ** 2 * 1e-5 * np.abs(a0).max()
        assert np.abs(xg[off[c]:off[c + 1]] - xs[-1]).max() <= bound


def _ragged_ensemble(zero_eps: bool):
    """Clusters of 1 ... 5000 particles: single particles, exact tiles, tiles plus one, several i-blocks,
    several j tiles; with zero_eps one cluster has eps = 0 (the guarded pair arithmetic for the batch)."""
    sizes = [1, 2, 127, 128, 129, 300, 513, 1000, 2049, 5000]
    clusters = [workloads.plummer(n, (321, c), eps=1.0 / 128 if n > 1 else 0.01) for c, n in enumerate(sizes)]
    if zero_eps:
        clusters[6].eps = 0.0
    off = np.concatenate([[0], np.cumsum(sizes)])
    m = np.concatenate([c.m for c in clusters])
    x = np.concatenate([c.x for c in clusters])
    v = np.concatenate([c.v for c in clusters])
    return clusters, off, m, x, v


@pytest.mark.parametrize("zero_eps", [False, True])
def test_batched_decompositions_match_oracle(kirin_lib, zero_eps):
    """Every work decomposition (512, 256 or 128 i per item; whole clusters or j ranges of 1, 2, 3 or
    16 tiles, which splits every cluster with more than that many tiles) against the oracle, and the
    same decomposition twice bit for bit (the split sums are added in a fixed order)."""
    clusters, off, m, x, v = _ragged_ensemble(zero_eps)
    refs = [oracle.acc_pot(cl.m, cl.x, cl.eps)[0] for cl in clusters]  # eps = 0: no coincident pairs here
    b = abi.KirinBatch(off, [c.eps for c in clusters])
    assert b.get_launch()[:2] == (1, 0)
    for bad in ((3, 0), (8, 0), (1, -1)):
        with pytest.raises(abi.KirinError):
            b.set_launch(*bad)
    assert b.get_launch()[:2] == (1, 0)
    for groups, j_tiles in ((1, 0), (2, 0), (4, 0), (1, 1), (2, 2), (4, 3), (1, 16), (4, 1)):
        b.set_launch(groups, j_tiles)
        assert b.get_launch()[:2] == (groups, j_tiles)
        b.set_state(m, x, v)
        acc = b.accel()
        again = b.accel()
        assert np.array_equal(acc, again), (groups, j_tiles)
        for c, cl in enumerate(clusters):
            if cl.n == 1:
                assert np.all(acc[off[c]:off[c + 1]] == 0.0)
                continue
            e = metrics.rel_err_vec(acc[off[c]:off[c + 1]], refs[c])
            assert np.median(e) <= 1e-6 and e.max() <= 1e-5, (groups, j_tiles, c, np.median(e), e.max())
    b.close()


def test_batched_split_leapfrog_graph_is_identical(kirin_lib):
    """With split j ranges the captured graph replays the eager launches bit for bit."""
    clusters, off, m, x, v = _ragged_ensemble(False)
    finals = []
    for use_graph in (False, True):
        b = abi.KirinBatch(off, [c.eps for c in clusters])
        b.set_launch(2, 2)
        b.set_state(m, x, v)
        b.leapfrog(1.0 / 256, 6, use_graph=use_graph)
        b.leapfrog(1.0 / 256, 6, use_graph=use_graph)  # a replay of the captured graph
        b.sync()
        finals.append(b.get_state())
        b.close()
    assert np.array_equal(finals[0][0], finals[1][0]) and np.array_equal(finals[0][1], finals[1][1])


def test_batch_tuner_installs_a_timed_decomposition(kirin_lib):
    from paper_0707_0438_gb300 import autotune
    clusters, off, m, x, v = _ragged_ensemble(False)
    b = abi.KirinBatch(off, [c.eps for c in clusters])
    g, jt, timed = autotune.tune_batch(b, m, x, v, candidates=((1, 0), (2, 0), (4, 4)))
    assert {(e[0], e[1]) for e in timed} == {(1, 0), (2, 0), (4, 4)} and all(e[2] > 0 for e in timed)
    assert (g, jt) in {(e[0], e[1]) for e in timed} and b.get_launch()[:2] == (g, jt)
    acc = b.accel()  # the state was put back
    b.close()
    ra, _ = oracle.acc_pot(clusters[-1].m, clusters[-1].x, clusters[-1].eps)
    assert metrics.rel_err_vec(acc[off[-2]:off[-1]], ra).max() <= 1e-5


def test_batch_with_empty_clusters(kirin_lib):
    """Clusters of zero particles (repeated offsets) own no work items and leave their neighbours intact."""
    a = workloads.plummer(5, (55, 1), eps=0.05)
    b_ = workloads.plummer(300, (55, 2), eps=0.01)
    off = np.array([0, 0, 5, 5, 305, 305])
    eps = [0.1, a.eps, 0.1, b_.eps, 0.1]
    m, x, v = (np.concatenate([getattr(a, k), getattr(b_, k)]) for k in ("m", "x", "v"))
    with abi.KirinBatch(off, eps) as b:
        for groups, j_tiles in ((1, 0), (4, 1)):
            b.set_launch(groups, j_tiles)
            b.set_state(m, x, v)
            acc = b.accel()
            for cl, lo, hi in ((a, 0, 5), (b_, 5, 305)):
                ra, _ = oracle.acc_pot(cl.m, cl.x, cl.eps)
                e = metrics.rel_err_vec(acc[lo:hi], ra)
                assert np.median(e) <= 1e-6 and e.max() <= 1e-5, (groups, j_tiles, e.max())
    assert b.b is None


def test_batch_device_pointer_twins(kirin_lib):
    """set_state_dev / accel_dev / get_state_dev give the host path's results bit for bit; accel before
    any state is ESTATE; a non-finite upload is reported by the next sync."""
    import torch
    clusters, off, m, x, v = _ragged_ensemble(False)
    dev = torch.device("cuda:0")
    md, xd, vd = (torch.tensor(a, device=dev) for a in (m, x, v))
    torch.cuda.synchronize()  # the batch enqueues on a stream of its own
    with abi.KirinBatch(off, [c.eps for c in clusters]) as b:
        b.set_launch(2, 2)
        b.set_state(m, x, v)
        acc_host = b.accel()
        b.leapfrog(1.0 / 256, 3, use_graph=False)
        b.sync()
        x_host, v_host = b.get_state()
    with abi.KirinBatch(off, [c.eps for c in clusters]) as b:
        acc = torch.empty_like(xd)
        with pytest.raises(abi.KirinError) as e:
            b.accel_dev(acc)
        assert e.value.code == abi.KIRIN_ESTATE
        with pytest.raises(ValueError):
            b.accel_dev(torch.empty((b.n_total, 3), dtype=torch.float32, device=dev))
        b.set_launch(2, 2)
        b.set_state_dev(md, xd, vd)
        b.accel_dev(acc)
        b.leapfrog(1.0 / 256, 3, use_graph=False)
        xo, vo = torch.empty_like(xd), torch.empty_like(vd)
        b.get_state_dev(xo, vo)
        b.sync()
        assert np.array_equal(acc.cpu().numpy(), acc_host)
        assert np.array_equal(xo.cpu().numpy(), x_host) and np.array_equal(vo.cpu().numpy(), v_host)
        bad = vd.clone()
        bad[5, 1] = float("nan")
        torch.cuda.synchronize()
        b.set_state_dev(md, xd, bad)
        with pytest.raises(abi.KirinError) as e:
            b.sync()
        assert e.value.code == abi.KIRIN_ENONFINITE
