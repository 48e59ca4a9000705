"""4th-order Hermite predictor-corrector with shared or block time-steps -- TEST INFRASTRUCTURE.

Sect. 3 of the paper names the scheme (Makino & Aarseth 1992: predictor,
Hermite interpolation, corrector; block time-steps after Makino 1991) and
splits it so that prediction and correction run in FP64 on the host while the
direct sum (acc, jerk, pot) runs on the accelerator.  The formulas are not
printed in the paper; the ones below are the standard scheme:

  predictor  x_p = x + v dt + a dt^2/2 + j dt^3/6,  v_p = v + a dt + j dt^2/2
  Hermite    a2 = [-6 (a0 - a1) - dt (4 j0 + 2 j1)] / dt^2
             a3 = [12 (a0 - a1) + 6 dt (j0 + j1)] / dt^3
  corrector  x1 = x_p + a2 dt^4/24 + a3 dt^5/120,  v1 = v_p + a2 dt^3/6 + a3 dt^4/24
  Aarseth    dt = sqrt(eta (|a1| |a2'| + |j1|^2) / (|j1| |a3| + |a2'|^2)),  a2' = a2 + dt a3

Block steps: dt is a power of two in [2^-20, 2^-3]; a step may shrink freely
but may only double when the new time is a multiple of the doubled step; the
block at each step is every particle with t_i + dt_i equal to the smallest such
sum.  The start-up step is 0.01 |a| / |j| quantised down.

The force evaluation is pluggable (``force(x, v, i_idx) -> (acc, jerk, pot)``);
by default it is the FP64 oracle.
"""
from __future__ import annotations

import math

import numpy as np

from . import acc_jerk_pot, energy

DT_MIN = 2.0 ** -20
DT_MAX = 2.0 ** -3


def predict(x, v, a, j, dt):
    """Taylor predictor to second (v) and third (x) order; dt is a scalar or an (n,) array."""
    dt = np.asarray(dt, dtype=np.float64)
    if dt.ndim == 1:
        dt = dt[:, None]
    xp = x + v * dt + a * (dt * dt / 2.0) + j * (dt * dt * dt / 6.0)
    vp = v + a * dt + j * (dt * dt / 2.0)
    return xp, vp


def hermite_derivatives(a0, j0, a1, j1, dt):
    """Second and third derivatives of a at the start of the step from the two (a, jerk) pairs."""
    dt = np.asarray(dt, dtype=np.float64)
    if dt.ndim == 1:
        dt = dt[:, None]
    a2 = (-6.0 * (a0 - a1) - dt * (4.0 * j0 + 2.0 * j1)) / (dt * dt)
    a3 = (12.0 * (a0 - a1) + 6.0 * dt * (j0 + j1)) / (dt * dt * dt)
    return a2, a3


def correct(xp, vp, a2, a3, dt):
    dt = np.asarray(dt, dtype=np.float64)
    if dt.ndim == 1:
        dt = dt[:, None]
    x1 = xp + a2 * dt ** 4 / 24.0 + a3 * dt ** 5 / 120.0
    v1 = vp + a2 * dt ** 3 / 6.0 + a3 * dt ** 4 / 24.0
    return x1, v1


def aarseth_step(a1, j1, a2, a3, dt, eta):
    """Aarseth's criterion evaluated at the end of the step (a2 carried to t1)."""
    dt = np.asarray(dt, dtype=np.float64)
    dtc = dt[:, None] if dt.ndim == 1 else dt
    a2e = a2 + dtc * a3
    na = np.linalg.norm(a1, axis=1)
    nj = np.linalg.norm(j1, axis=1)
    n2 = np.linalg.norm(a2e, axis=1)
    n3 = np.linalg.norm(a3, axis=1)
    return np.sqrt(eta * (na * n2 + nj * nj) / (nj * n3 + n2 * n2))


def quantise_initial(dt_raw):
    """Largest power of two <= dt_raw, clamped to [DT_MIN, DT_MAX]."""
    out = np.empty_like(dt_raw)
    for k, d in enumerate(dt_raw):
        q = DT_MAX
        while q > d and q > DT_MIN:
            q *= 0.5
        out[k] = q
    return out


def next_step(dt_old, dt_raw, t_new):
    """Power-of-two block step update: shrink freely, double only on a commensurate time."""
    out = np.empty_like(dt_old)
    for k in range(dt_old.shape[0]):
        d_old, d_raw = dt_old[k], dt_raw[k]
        if d_raw < d_old:
            q = d_old
            while q > d_raw and q > DT_MIN:
                q *= 0.5
        elif d_raw >= 2.0 * d_old and 2.0 * d_old <= DT_MAX and math.fmod(t_new, 2.0 * d_old) == 0.0:
            q = 2.0 * d_old
        else:
            q = d_old
        out[k] = min(max(q, DT_MIN), DT_MAX)
    return out


def _oracle_force(m, eps, G):
    def force(x, v, i_idx):
        return acc_jerk_pot(m, x, v, eps, G, i_idx=i_idx)
    return force


def shared_steps(m, x, v, eps, dt, n_steps, G=1.0, force=None):
    """n_steps Hermite steps with one shared dt for all particles.

    Returns (x, v, a, j) after the last step and the list of (acc, jerk, pot) of every evaluation.
    """
    force = force or _oracle_force(m, eps, G)
    n = m.shape[0]
    idx = np.arange(n)
    a, j, pot = force(x, v, idx)
    evals = [(a, j, pot)]
    for _ in range(n_steps):
        xp, vp = predict(x, v, a, j, dt)
        a1, j1, pot1 = force(xp, vp, idx)
        a2, a3 = hermite_derivatives(a, j, a1, j1, dt)
        x, v = correct(xp, vp, a2, a3, dt)
        a, j = a1, j1
        evals.append((a1, j1, pot1))
    return x, v, a, j, evals


def block_steps(m, x, v, eps, t_end, eta=0.01, G=1.0, force=None, max_steps=None):
    """Block time-step Hermite integration from t = 0 to t_end (a multiple of DT_MAX).

    Returns a dict with the final state, the list of active-block sizes and the
    energies at start and end (Eq. 2).
    """
    force = force or _oracle_force(m, eps, G)
    n = m.shape[0]
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    idx_all = np.arange(n)
    a, j, _ = force(x, v, idx_all)
    t = np.zeros(n)
    dt = quantise_initial(0.01 * np.linalg.norm(a, axis=1) / np.linalg.norm(j, axis=1))
    e0 = sum(energy(m, x, v, eps, G))
    blocks = []
    steps = 0
    while True:
        t_next = float(np.min(t + dt))
        if t_next > t_end:
            break
        act = np.nonzero(t + dt == t_next)[0]
        xp, vp = predict(x, v, a, j, t_next - t)
        a1, j1, _ = force(xp, vp, act)
        h = dt[act]
        a2, a3 = hermite_derivatives(a[act], j[act], a1, j1, h)
        x1, v1 = correct(xp[act], vp[act], a2, a3, h)
        dt_raw = aarseth_step(a1, j1, a2, a3, h, eta)
        dt[act] = next_step(h, dt_raw, t_next)
        x[act], v[act], a[act], j[act] = x1, v1, a1, j1
        t[act] = t_next
        blocks.append(act.shape[0])
        steps += 1
        if max_steps is not None and steps >= max_steps:
            break
    e1 = sum(energy(m, x, v, eps, G))
    return {"x": x, "v": v, "a": a, "j": j, "t": t, "dt": dt, "blocks": blocks,
            "e_start": e0, "e_end": e1, "dE_E": (e0 - e1) / e0}
