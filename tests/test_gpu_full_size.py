"""The secondary workloads at their full sizes, in the launch configuration the benchmark times:
sampled outputs against the FP64 oracle where it can keep up, properties that hold at any size
otherwise (energy, the block-time grid, a directional derivative of the adjoint)."""
import numpy as np
import pytest

import oracle
from paper_0707_0438_gb300 import abi, autotune, metrics, workloads
from tests.gpu_util import assert_parity

pytestmark = pytest.mark.gpu


def test_ensemble_full_size_sampled_parity(kirin_lib):
    """512 clusters (N_c log-uniform in [256, 16384), eps = 1/N_c) in one batched launch, in the
    decomposition the tuner picks (as the benchmark does): the largest, the smallest and two random
    clusters against the oracle, every particle."""
    clusters, sizes = workloads.ensemble()
    off = np.concatenate([[0], np.cumsum(sizes)])
    m, x, v = (np.concatenate([getattr(c, a) for c in clusters]) for a in ("m", "x", "v"))
    b = abi.KirinBatch(off, [c.eps for c in clusters])
    autotune.tune_batch(b, m, x, v)
    acc = b.accel()
    b.close()
    rng = np.random.default_rng(11)
    pick = {int(np.argmax(sizes)), int(np.argmin(sizes))} | set(rng.choice(len(sizes), 2, replace=False).tolist())
    for c in sorted(pick):
        cl = clusters[c]
        ra, _ = oracle.acc_pot(cl.m, cl.x, cl.eps)
        e = metrics.rel_err_vec(acc[off[c]:off[c + 1]], ra)
        assert np.median(e) <= 1e-6 and e.max() <= 1e-5, (c, sizes[c], np.median(e), e.max())


def _block_ctx(p, device_loop):
    import torch
    k = abi.Kirin(p.n, p.eps, precision="mixed")
    k.set_j_particles(p.m, p.x, p.v)
    autotune.install(k, p.n, torch.cuda.get_device_name(0), "mixed")
    k.set_device_loop(device_loop)
    return k


def test_block_workload_full_size(kirin_lib):
    """N = 65536, eps = 1e-3 with the packaged launch table: the starting evaluation on sampled i
    against the oracle, then block steps to t = 1/64 by the device loop: energy conserved, every
    particle on the block-time grid, the host loop's schedule."""
    p = workloads.config_block(65536)
    t_end = 1.0 / 64
    il = workloads.i_subset(p.n, 256, seed=9)
    with _block_ctx(p, True) as k:
        start = k.forces(il)  # the block-start evaluation of the sampled i: acc, jerk and pot
        e0 = sum(k.energy())
        k.hermite_init(0.0)
        st0 = k.get_state()
        steps, pairs = k.hermite_run(t_end)
        st = k.get_state()
        e1 = sum(k.energy())
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    assert_parity(start, ref, "mixed", "block start, sampled i")
    # hermite_init's own evaluation of every particle holds the same acc and jerk for those i
    assert_parity((st0["a"][il], st0["j"][il], start[2]), ref, "mixed", "block start, state")
    assert steps > 100 and pairs >= steps * p.n
    assert abs(metrics.energy_error(e0, e1)) < 1e-6
    t, dt = st["t"], st["dt"]
    assert np.all(t <= t_end) and np.all(t + dt > t_end)
    assert np.all((dt >= 2.0 ** -20) & (dt <= 2.0 ** -3))
    assert np.all(np.frexp(dt)[0] == 0.5)  # powers of two
    assert np.all(np.mod(t, dt) == 0.0)     # commensurate: each particle sits on its own level's grid
    with _block_ctx(p, False) as k:
        k.hermite_init(0.0)
        host_steps, _ = k.hermite_run(t_end)
        sh = k.get_state()
    assert abs(host_steps - steps) <= 2
    assert np.abs(sh["x"] - st["x"]).max() <= 1e-9 * np.abs(p.x).max()


def test_adjoint_full_size_directional_derivative(kirin_lib):
    """N = 16384, eps = 0.01, 64 leapfrog steps of 1/128 with checkpoints every 8 (the benchmark's
    configuration) in FP64: the checkpointed adjoint gradient along a random direction equals the
    central difference of the loss."""
    import torch
    from paper_0707_0438_gb300 import autograd as kag
    dev = torch.device("cuda:0")
    p = workloads.config_adjoint(16384)
    q = workloads.perturb(p, 1e-3)
    dt, steps = 1.0 / 128, 64
    rng = np.random.default_rng(12)
    dx = rng.standard_normal(p.x.shape)
    dx /= np.linalg.norm(dx)
    with abi.Kirin(p.n, p.eps, precision="fp64", stream=torch.cuda.current_stream().cuda_stream) as k:
        tgt = torch.tensor(q.x, device=dev)
        v = torch.tensor(p.v, device=dev)
        m = torch.tensor(p.m, device=dev)

        def loss(x):
            xf, _ = kag.leapfrog(x, v, m, k, dt, steps, every=8)
            return ((xf - tgt) ** 2).sum(dim=1).mean()

        x = torch.tensor(p.x, device=dev, requires_grad=True)
        L = loss(x)
        L.backward()
        g_dir = float((x.grad * torch.tensor(dx, device=dev)).sum())
        h = 1e-5
        with torch.no_grad():
            lp = float(loss(torch.tensor(p.x + h * dx, device=dev)))
            lm = float(loss(torch.tensor(p.x - h * dx, device=dev)))
    fd = (lp - lm) / (2 * h)
    assert np.isfinite(g_dir) and g_dir != 0.0
    assert abs(fd - g_dir) <= 1e-4 * abs(g_dir), (fd, g_dir)


def test_adjoint_workload_calls_full_size_match_oracle(kirin_lib):
    """The two force calls of the differentiable leapfrog at N = 16384 in the packaged launch shapes
    (acc + pot: 1 j-group x 32 splits; adjoint: 4 x 8, as the benchmark runs them), mixed precision,
    against the FP64 oracle for every particle."""
    import torch
    dev = torch.device("cuda:0")
    p = workloads.config_adjoint(16384)
    g = np.random.default_rng(21).standard_normal((p.n, 3))
    m, x, gt = (torch.tensor(a, device=dev) for a in (p.m, p.x, g))
    acc, gx = torch.empty_like(x), torch.empty_like(x)
    pot, gm = torch.empty_like(m), torch.empty_like(m)
    with abi.Kirin(p.n, p.eps, precision="mixed", stream=torch.cuda.current_stream().cuda_stream) as k:
        autotune.install(k, p.n, torch.cuda.get_device_name(0), "mixed")
        k.accel_dev(m, x, acc, pot)
        k.accel_adjoint_dev(m, x, gt, gx, gm)
        k.sync()
    ra, rp = oracle.acc_pot(p.m, p.x, p.eps)
    rgx, rgm = oracle.force_adjoint(p.m, p.x, g, p.eps)
    e = metrics.rel_err_vec(acc.cpu().numpy(), ra)
    assert np.median(e) <= 1e-6 and e.max() <= 1e-5, ("acc", np.median(e), e.max())
    e = metrics.rel_err_scalar(pot.cpu().numpy(), rp)
    assert np.median(e) <= 1e-6 and e.max() <= 1e-5, ("pot", np.median(e), e.max())
    # random-sign sums over j: the median per particle, the worst against the gradient's RMS size
    for name, got, ref in (("dL/dx", gx.cpu().numpy(), rgx), ("dL/dm", gm.cpu().numpy()[:, None], rgm[:, None])):
        err = np.linalg.norm(got - ref, axis=1)
        rms = np.sqrt(np.mean(np.sum(ref * ref, axis=1)))
        assert np.median(err / np.linalg.norm(ref, axis=1)) <= 1e-6 and err.max() / rms <= 1e-5, name
