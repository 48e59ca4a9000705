"""Throughput and error conventions used by the tests and the benchmark.

* Eq. 3: P = k N^2 / t, with k = 60 flops per interaction for acceleration +
  jerk + potential and k = 38 for the force alone (Sect. 4.1).  The paper
  counts all N^2 (i, j) pairs, self pairs included (Sect. 3.1).
* Eq. 2: dE/E = (E_start - E_end) / E_start.
* Per-particle relative error |q - q_ref| / |q_ref| (median and max), and the
  cancellation-free variant |da| / sum_j m_j / s_ij^2 for accelerations.
"""
from __future__ import annotations

import numpy as np

K_ACC_JERK_POT = 60
K_FORCE_ONLY = 38


def flops_per_second(n_i: float, n_j: float, seconds: float, k: int = K_ACC_JERK_POT) -> float:
    """k n_i n_j / t (Eq. 3; n_i = n_j = N for a full evaluation)."""
    return k * float(n_i) * float(n_j) / seconds


def interactions_per_second(n_i: float, n_j: float, seconds: float) -> float:
    return float(n_i) * float(n_j) / seconds


def energy_error(e_start: float, e_end: float) -> float:
    """Relative energy error of Eq. 2."""
    return (e_start - e_end) / e_start


def rel_err_vec(q, q_ref):
    """Per-row |q - q_ref| / |q_ref| for (n, 3) arrays."""
    q, q_ref = np.asarray(q, dtype=np.float64), np.asarray(q_ref, dtype=np.float64)
    return np.linalg.norm(q - q_ref, axis=1) / np.maximum(np.linalg.norm(q_ref, axis=1), 1e-300)


def rel_err_scalar(q, q_ref):
    q, q_ref = np.asarray(q, dtype=np.float64), np.asarray(q_ref, dtype=np.float64)
    return np.abs(q - q_ref) / np.maximum(np.abs(q_ref), 1e-300)


def summary(err) -> dict:
    err = np.asarray(err, dtype=np.float64)
    if err.size == 0:
        return {"median": 0.0, "max": 0.0}
    return {"median": float(np.median(err)), "max": float(np.max(err))}
