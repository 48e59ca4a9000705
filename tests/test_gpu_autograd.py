"""Differentiable accelerations and leapfrog trajectories: finite differences and the FP64 oracle gradient."""
import numpy as np
import pytest

import oracle
from oracle import leapfrog as olf
from paper_0707_0438_gb300 import abi, workloads

pytestmark = pytest.mark.gpu


def _t(a, dev, grad=False):
    import torch
    return torch.tensor(a, dtype=torch.float64, device=dev, requires_grad=grad)


def test_accel_gradcheck_fp64(kirin_lib):
    import torch
    from paper_0707_0438_gb300 import autograd as kag
    dev = torch.device("cuda:0")
    p = workloads.plummer(64, 1005, masses="lognormal", eps=0.05)
    with abi.Kirin(64, p.eps, precision="fp64", stream=torch.cuda.current_stream().cuda_stream) as k:
        x, m = _t(p.x, dev, True), _t(p.m, dev, True)
        assert torch.autograd.gradcheck(lambda xx, mm: kag.accel(xx, mm, k), (x, m), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_leapfrog_gradcheck_fp64(kirin_lib):
    """Config 5's checks at N = 64: the whole checkpointed trajectory against central differences."""
    import torch
    from paper_0707_0438_gb300 import autograd as kag
    dev = torch.device("cuda:0")
    p = workloads.plummer(64, 1005, eps=0.01)
    with abi.Kirin(64, p.eps, precision="fp64", stream=torch.cuda.current_stream().cuda_stream) as k:
        x, v, m = _t(p.x, dev, True), _t(p.v, dev, True), _t(p.m, dev, True)
        tgt = _t(p.x + 0.01, dev)

        def loss(xx, vv, mm):
            xf, _ = kag.leapfrog(xx, vv, mm, k, 1.0 / 128, 12, every=8)
            return ((xf - tgt) ** 2).sum(dim=1).mean()

        assert torch.autograd.gradcheck(loss, (x, v, m), eps=1e-6, atol=1e-8, rtol=1e-4)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_leapfrog_gradient_matches_oracle(kirin_lib, precision, tol):
    """Checkpointed GPU gradient against the FP64 CPU discrete adjoint (a shorter config-5 trajectory)."""
    import torch
    from paper_0707_0438_gb300 import autograd as kag
    dev = torch.device("cuda:0")
    n, steps, dt = 2048, 16, 1.0 / 128
    p = workloads.plummer(n, 1005, eps=0.01)
    q = workloads.perturb(p, 1e-3)
    xs, _ = olf.trajectory(q.m, q.x, q.v, q.eps, dt, steps)
    target = xs[-1]
    L_ref, gx_ref, gv_ref, gm_ref = olf.loss_grad(p.m, p.x, p.v, p.eps, dt, steps, target)
    with abi.Kirin(n, p.eps, precision=precision, stream=torch.cuda.current_stream().cuda_stream) as k:
        x, v, m = _t(p.x, dev, True), _t(p.v, dev, True), _t(p.m, dev, True)
        xf, _ = kag.leapfrog(x, v, m, k, dt, steps, every=8)
        L = ((xf - _t(target, dev)) ** 2).sum(dim=1).mean()
        L.backward()
    assert L.item() == pytest.approx(L_ref, rel=max(tol, 1e-12) * 100)
    for got, ref in ((x.grad, gx_ref), (v.grad, gv_ref), (m.grad, gm_ref)):
        err = np.linalg.norm(got.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= tol, err


@pytest.mark.slow
def test_leapfrog_gradient_full_config_mixed_matches_oracle(kirin_lib):
    """The differentiable-leapfrog workload as configured: N = 16384 Plummer sphere, eps = 0.01, 64
    KDK steps of dt = 1/128, checkpoints every 8, mixed-precision forward and adjoint kernels; loss =
    mean squared distance of the final positions to targets from the 1e-3-perturbed state.  The
    gradients with respect to x, v and m against the FP64 oracle's discrete adjoint: relative L2
    error <= 1e-5 and per-particle median <= 1e-5."""
    import torch
    from paper_0707_0438_gb300 import autograd as kag
    dev = torch.device("cuda:0")
    p = workloads.config_adjoint(16384)
    q = workloads.perturb(p, 1e-3)
    dt, steps = 1.0 / 128, 64
    xs, _ = olf.trajectory(q.m, q.x, q.v, q.eps, dt, steps)
    target = xs[-1]
    L_ref, gx_ref, gv_ref, gm_ref = olf.loss_grad(p.m, p.x, p.v, p.eps, dt, steps, target)
    with abi.Kirin(p.n, p.eps, precision="mixed", stream=torch.cuda.current_stream().cuda_stream) as k:
        x, v, m = _t(p.x, dev, True), _t(p.v, dev, True), _t(p.m, dev, True)
        xf, _ = kag.leapfrog(x, v, m, k, dt, steps, every=8)
        L = ((xf - _t(target, dev)) ** 2).sum(dim=1).mean()
        L.backward()
    assert L.item() == pytest.approx(L_ref, rel=1e-5)
    for name, got, ref in (("x", x.grad, gx_ref), ("v", v.grad, gv_ref), ("m", m.grad, gm_ref[:, None])):
        got = got.cpu().numpy().reshape(ref.shape)
        rel_l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        per = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert rel_l2 <= 1e-5 and np.median(per) <= 1e-5, (name, rel_l2, np.median(per), per.max())
