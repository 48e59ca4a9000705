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


def _trajectory_grads(p, target, dt, steps, precision):
    import torch
    from paper_0707_0438_gb300 import autograd as kag
    dev = torch.device("cuda:0")
    with abi.Kirin(p.n, p.eps, precision=precision, stream=torch.cuda.current_stream().cuda_stream) as k:
        x, v, m = _t(p.x, dev, True), _t(p.v, dev, True), _t(p.m, dev, True)
        xf, _ = kag.leapfrog(x, v, m, k, dt, steps, every=8)
        L = ((xf - _t(target, dev)) ** 2).sum(dim=1).mean()
        L.backward()
    return L.item(), x.grad.cpu().numpy(), v.grad.cpu().numpy(), m.grad.cpu().numpy()[:, None]


def _grad_errors(got, ref):
    """(relative L2 error, per-particle median relative error) of each of dL/dx, dL/dv, dL/dm."""
    out = {}
    for name, g, r in zip(("x", "v", "m"), got, ref):
        out[name] = (np.linalg.norm(g - r) / np.linalg.norm(r),
                     np.median(np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)))
    return out


@pytest.mark.slow
def test_leapfrog_gradient_full_config_matches_oracle(kirin_lib):
    """The differentiable-leapfrog workload as configured: N = 16384 Plummer sphere, eps = 0.01, 64
    KDK steps of dt = 1/128, checkpoints every 8; loss = mean squared distance of the final positions
    to targets from the 1e-3-perturbed state.  Gradients with respect to x, v and m against the FP64
    oracle's discrete adjoint.

    FP64 kernels: relative L2 and per-particle median errors <= 1e-10.  Mixed precision (FP32 pair
    arithmetic in the forward and the adjoint kernels): <= 1e-5 for dL/dx and dL/dv.  dL/dm sums a
    contribution of every one of the 65 adjoint calls, and its error grows with the length of the
    trajectory as the others do, about fivefold per doubling of the step count (measured on GB300:
    relative L2 4.5e-7, 9.4e-6, 4.5e-5 after 8, 32, 64 steps), while a single adjoint call stays at
    2e-7 at any step.  The growth is the trajectory's sensitivity to the FP32 rounding of the forward
    forces (the FP64 kernels on the same trajectory agree to 1e-13), so the mixed dL/dm is held to
    2e-4 (relative L2) and 1e-4 (median) at 64 steps, and to 2e-6 for all three after 8 steps."""
    p = workloads.config_adjoint(16384)
    q = workloads.perturb(p, 1e-3)
    dt = 1.0 / 128
    for steps in (8, 64):
        xs, _ = olf.trajectory(q.m, q.x, q.v, q.eps, dt, steps)
        target = xs[-1]
        L_ref, gx_ref, gv_ref, gm_ref = olf.loss_grad(p.m, p.x, p.v, p.eps, dt, steps, target)
        ref = (gx_ref, gv_ref, gm_ref[:, None])
        precisions = ("fp64", "mixed") if steps == 64 else ("mixed",)
        for precision in precisions:
            L, *got = _trajectory_grads(p, target, dt, steps, precision)
            errs = _grad_errors(got, ref)
            if precision == "fp64":
                assert L == pytest.approx(L_ref, rel=1e-12)
                bounds = {"x": (1e-10, 1e-10), "v": (1e-10, 1e-10), "m": (1e-10, 1e-10)}
            elif steps == 8:
                assert L == pytest.approx(L_ref, rel=1e-6)
                bounds = {"x": (2e-6, 2e-6), "v": (2e-6, 2e-6), "m": (2e-6, 2e-6)}
            else:
                assert L == pytest.approx(L_ref, rel=1e-5)
                bounds = {"x": (1e-5, 1e-5), "v": (1e-5, 1e-5), "m": (2e-4, 1e-4)}
            for name, (l2, med) in errs.items():
                assert l2 <= bounds[name][0] and med <= bounds[name][1], (steps, precision, name, l2, med)
