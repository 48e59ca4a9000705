"""CPU oracle for the direct N-body hot path (FP64) -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg and
reference arm may import this package.  It shares no code with the CUDA
library and never imports it.

* ``acc_jerk_pot`` / ``acc_pot`` / ``energy`` / ``force_adjoint`` / ``nearest``:
  thin ctypes wrappers over kirin_oracle.c (plain FP64 C, OpenMP over i).
* ``oracle.hermite``: 4th-order Hermite predictor-corrector with shared and
  block time-steps (Sect. 3, Makino & Aarseth 1992), numpy.
* ``oracle.leapfrog``: kick-drift-kick leapfrog (Sect. 4.3) and its discrete
  adjoint, numpy.

Parity pins for every function live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64, dbl = ctypes.c_int64, ctypes.c_double
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_acc_jerk_pot.argtypes = [i64, _ip, i64, _dp, _dp, _dp, dbl, dbl, dbl, _dp, _dp, _dp]
        lib.oracle_acc_pot.argtypes = [i64, _ip, i64, _dp, _dp, dbl, dbl, _dp, _dp]
        lib.oracle_energy.argtypes = [i64, _dp, _dp, _dp, dbl, dbl, _dp, _dp]
        lib.oracle_force_adjoint.argtypes = [i64, _dp, _dp, _dp, dbl, dbl, _dp, _dp]
        lib.oracle_nearest.argtypes = [i64, _ip, i64, _dp, _ip, _dp]
        for f in (lib.oracle_acc_jerk_pot, lib.oracle_acc_pot, lib.oracle_energy,
                  lib.oracle_force_adjoint, lib.oracle_nearest):
            f.restype = None
        _lib = lib
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _idx(i_idx, n):
    if i_idx is None:
        return np.arange(n, dtype=np.int64)
    i_idx = np.ascontiguousarray(i_idx, dtype=np.int64)
    if i_idx.size and (i_idx.min() < 0 or i_idx.max() >= n):
        raise IndexError("i index out of range")
    return i_idx


def num_threads() -> int:
    """OpenMP threads the oracle runs on (OMP_NUM_THREADS, else all host cores)."""
    return int(_load().oracle_num_threads())


def acc_jerk_pot(m, x, v, eps, G=1.0, i_idx=None, r_min=0.0):
    """Softened acceleration, jerk and potential of the i-particles (default: all) against all j != i."""
    lib = _load()
    m, x, v = _d(m), _d(x), _d(v)
    n = m.shape[0]
    idx = _idx(i_idx, n)
    k = idx.shape[0]
    acc = np.zeros((k, 3))
    jerk = np.zeros((k, 3))
    pot = np.zeros(k)
    lib.oracle_acc_jerk_pot(k, idx.ctypes.data_as(_ip), n, _p(m), _p(x), _p(v),
                            float(eps), float(r_min), float(G), _p(acc), _p(jerk), _p(pot))
    return acc, jerk, pot


def acc_pot(m, x, eps, G=1.0, i_idx=None):
    """Softened acceleration and potential (no jerk)."""
    lib = _load()
    m, x = _d(m), _d(x)
    n = m.shape[0]
    idx = _idx(i_idx, n)
    k = idx.shape[0]
    acc = np.zeros((k, 3))
    pot = np.zeros(k)
    lib.oracle_acc_pot(k, idx.ctypes.data_as(_ip), n, _p(m), _p(x), float(eps), float(G),
                       _p(acc), _p(pot))
    return acc, pot


def energy(m, x, v, eps, G=1.0):
    """(K, W): kinetic energy and softened potential energy 1/2 sum m_i phi_i."""
    lib = _load()
    m, x, v = _d(m), _d(x), _d(v)
    kin = ctypes.c_double()
    pot = ctypes.c_double()
    lib.oracle_energy(m.shape[0], _p(m), _p(x), _p(v), float(eps), float(G),
                      ctypes.byref(kin), ctypes.byref(pot))
    return kin.value, pot.value


def force_adjoint(m, x, g, eps, G=1.0):
    """(dL/dx, dL/dm) for L with dL/da = g, a = softened acceleration of all particles."""
    lib = _load()
    m, x, g = _d(m), _d(x), _d(g)
    n = m.shape[0]
    gx = np.zeros((n, 3))
    gm = np.zeros(n)
    lib.oracle_force_adjoint(n, _p(m), _p(x), _p(g), float(eps), float(G), _p(gx), _p(gm))
    return gx, gm


def nearest(x, i_idx=None):
    """(index, r^2) of the nearest j != i for each i-particle (smallest j on ties)."""
    lib = _load()
    x = _d(x)
    n = x.shape[0]
    idx = _idx(i_idx, n)
    k = idx.shape[0]
    nn = np.zeros(k, dtype=np.int64)
    r2 = np.zeros(k)
    lib.oracle_nearest(k, idx.ctypes.data_as(_ip), n, _p(x), nn.ctypes.data_as(_ip), _p(r2))
    return nn, r2
