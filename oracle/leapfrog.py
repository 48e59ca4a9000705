"""Kick-drift-kick leapfrog and its discrete adjoint, FP64 -- TEST INFRASTRUCTURE.

Sect. 4.3 of the paper drives the force library from a 2nd-order leapfrog with
a shared step and acceleration only.  One step of size dt, h = dt / 2:

  v_h = v + h a(x);   x' = x + dt v_h;   v' = v_h + h a(x')

The adjoint below is the chain rule applied to exactly these operations in
reverse order (the paper has no adjoint).  With (lx', lv') = dL/d(x', v'):

  lv_h = lv';  lx' += J(x')^T (h lv');  lm += M(x')^T (h lv')
  lx = lx';    lv_h += dt lx'
  lv = lv_h;   lx += J(x)^T (h lv_h);   lm += M(x)^T (h lv_h)

where J^T g and M^T g are the oracle's force_adjoint (dL/dx, dL/dm for dL/da = g).
"""
from __future__ import annotations

import numpy as np

from . import acc_pot, force_adjoint


def _acc(m, x, eps, G):
    a, _ = acc_pot(m, x, eps, G)
    return a


def trajectory(m, x0, v0, eps, dt, n_steps, G=1.0):
    """Run n_steps KDK steps; returns the list of positions and velocities (n_steps + 1 each)."""
    x, v = np.array(x0, dtype=np.float64), np.array(v0, dtype=np.float64)
    h = 0.5 * dt
    a = _acc(m, x, eps, G)
    xs, vs = [x.copy()], [v.copy()]
    for _ in range(n_steps):
        v = v + h * a
        x = x + dt * v
        a = _acc(m, x, eps, G)
        v = v + h * a
        xs.append(x.copy())
        vs.append(v.copy())
    return xs, vs


def loss(m, x0, v0, eps, dt, n_steps, target, G=1.0):
    """Mean over particles of the squared distance of the final positions to the targets."""
    xs, _ = trajectory(m, x0, v0, eps, dt, n_steps, G)
    d = xs[-1] - target
    return float(np.mean(np.sum(d * d, axis=1)))


def loss_grad(m, x0, v0, eps, dt, n_steps, target, G=1.0):
    """(L, dL/dx0, dL/dv0, dL/dm) by the discrete adjoint of the KDK steps."""
    m = np.asarray(m, dtype=np.float64)
    xs, vs = trajectory(m, x0, v0, eps, dt, n_steps, G)
    n = m.shape[0]
    h = 0.5 * dt
    d = xs[-1] - target
    L = float(np.mean(np.sum(d * d, axis=1)))
    lx = 2.0 * d / n
    lv = np.zeros_like(lx)
    lm = np.zeros(n)
    for k in range(n_steps - 1, -1, -1):
        x_k, x_k1 = xs[k], xs[k + 1]
        lvh = lv.copy()
        gx, gm = force_adjoint(m, x_k1, h * lv, eps, G)
        lx = lx + gx
        lm = lm + gm
        lvh = lvh + dt * lx
        gx, gm = force_adjoint(m, x_k, h * lvh, eps, G)
        lx = lx + gx
        lm = lm + gm
        lv = lvh
    return L, lx, lv, lm
