"""torch.autograd wrappers over libkirin: differentiable accelerations and
leapfrog trajectories with step checkpointing.

Argument marshalling only.  The forward force is kirin_accel_dev (FP32 pair
arithmetic on double-single positions for a mixed-precision context, FP64 for
an FP64 one), the backward is the hand-written adjoint kernel
(kirin_accel_adjoint_dev), and the leapfrog steps and their reverse sweep run
in kirin_leapfrog_dev / kirin_leapfrog_adjoint_dev.  The paper has no
adjoint; the leapfrog is the shared-step integrator of Sect. 4.3.

All tensors are float64 CUDA tensors: x, v (n, 3), m (n).  The context must
run on the current torch stream: create it with
stream=torch.cuda.current_stream().cuda_stream (0, torch's default stream, is
passed on as the legacy default stream).
"""
from __future__ import annotations

import torch

from .abi import Kirin


class KirinAccel(torch.autograd.Function):
    """a(x, m): softened accelerations of every particle; backward gives dL/dx and dL/dm."""

    @staticmethod
    def forward(ctx, x, m, kir: Kirin):
        x = x.contiguous()
        m = m.contiguous()
        acc = torch.empty_like(x)
        kir.accel_dev(m, x, acc)
        ctx.save_for_backward(x, m)
        ctx.kir = kir
        return acc

    @staticmethod
    def backward(ctx, g):
        x, m = ctx.saved_tensors
        gx = torch.empty_like(x)
        gm = torch.empty_like(m)
        ctx.kir.accel_adjoint_dev(m, x, g.contiguous(), gx, gm)
        return gx, gm, None


def accel(x, m, kir: Kirin):
    return KirinAccel.apply(x, m, kir)


class LeapfrogTrajectory(torch.autograd.Function):
    """(x_N, v_N) after n_steps KDK steps from (x0, v0); positions and
    velocities are checkpointed every `every` steps and each segment is
    recomputed during the reverse sweep."""

    @staticmethod
    def forward(ctx, x0, v0, m, kir: Kirin, dt: float, n_steps: int, every: int):
        x = x0.detach().clone().contiguous()
        v = v0.detach().clone().contiguous()
        m = m.detach().contiguous()
        acc = torch.empty_like(x)
        segs = []
        done = 0
        while done < n_steps:
            steps = min(every, n_steps - done)
            segs.append((x.clone(), v.clone(), steps))
            kir.leapfrog_dev(m, x, v, acc, dt, steps, acc_valid=done > 0)
            done += steps
        ctx.kir = kir
        ctx.dt = dt
        ctx.steps = [s for _, _, s in segs]
        ctx.save_for_backward(m, *[t for s in segs for t in s[:2]])
        return x, v

    @staticmethod
    def backward(ctx, gx, gv):
        m, *ck = ctx.saved_tensors
        n = m.shape[0]
        lx = gx.detach().clone().contiguous() if gx is not None else torch.zeros((n, 3), dtype=m.dtype, device=m.device)
        lv = gv.detach().clone().contiguous() if gv is not None else torch.zeros_like(lx)
        lm = torch.zeros_like(m)
        nseg = len(ctx.steps)
        for s in range(nseg - 1, -1, -1):
            steps = ctx.steps[s]
            x = ck[2 * s].clone()
            v = ck[2 * s + 1].clone()
            acc = torch.empty_like(x)
            hist = torch.empty((steps + 1, n, 3), dtype=m.dtype, device=m.device)
            ctx.kir.leapfrog_dev(m, x, v, acc, ctx.dt, steps, acc_valid=False, x_hist=hist)
            flags = (1 if s == nseg - 1 else 0) | (2 if s == 0 else 0)
            ctx.kir.leapfrog_adjoint_dev(m, hist, steps, ctx.dt, lx, lv, lm, flags)
        return lx, lv, lm, None, None, None, None


def leapfrog(x0, v0, m, kir: Kirin, dt: float, n_steps: int, every: int = 8):
    """Differentiable KDK trajectory; returns (x_N, v_N)."""
    return LeapfrogTrajectory.apply(x0, v0, m, kir, float(dt), int(n_steps), int(every))
