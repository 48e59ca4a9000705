"""Thin Python binding of libkirin's C ABI (include/kirin.h), via ctypes.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep their C names (``kirin_init``, ``kirin_compute_forces``
...) on the object returned by :func:`lib`; :class:`Kirin` and
:class:`KirinBatch` wrap a context with numpy (host) and torch (device)
arrays.  There is no fallback: if libkirin.so has not been built (see
``paper_0707_0438_gb300.build``), :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

KIRIN_OK = 0
KIRIN_EINVAL = -1
KIRIN_ENOMEM = -2
KIRIN_ECUDA = -3
KIRIN_ENONFINITE = -4
KIRIN_ETIMEOUT = -5
KIRIN_ESTATE = -6
KIRIN_EEXCHANGE = -7
KIRIN_FP64 = 0
KIRIN_MIXED = 1
# kirin_call_kind: the force calls that each have their own launch table
KIRIN_CALL_FORCES = 0
KIRIN_CALL_ACC_POT = 1
KIRIN_CALL_ADJOINT = 2
CALL_KINDS = {"forces": KIRIN_CALL_FORCES, "acc_pot": KIRIN_CALL_ACC_POT, "adjoint": KIRIN_CALL_ADJOINT}

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kirin.h")


class KirinError(RuntimeError):
    def __init__(self, code, what, detail=""):
        self.code = code
        super().__init__(f"{what}: {code} ({_strerror(code)}){' - ' + detail if detail else ''}")


class kirin_config(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("G", ctypes.c_double), ("r_min", ctypes.c_double),
                ("prec", ctypes.c_int32), ("device", ctypes.c_int32), ("stream", ctypes.c_void_p)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PI64 = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); pointers to device memory are passed as void*.
_SIGS = {
    "kirin_init": (ctypes.c_int, [ctypes.POINTER(_P), _I64, ctypes.POINTER(kirin_config)]),
    "kirin_finalize": (ctypes.c_int, [_P]),
    "kirin_query": (ctypes.c_int, [_P, _PI64, _PI32, _PI32]),
    "kirin_set_params": (ctypes.c_int, [_P, _D, _D, _D, _I32]),
    "kirin_set_stream": (ctypes.c_int, [_P, _P]),
    "kirin_set_launch": (ctypes.c_int, [_P, _I32, _I32]),
    "kirin_set_launch_table_for": (ctypes.c_int, [_P, _I32, _I32, _PI64, _PI32, _PI32]),
    "kirin_get_launch_for": (ctypes.c_int, [_P, _I32, _I64, _PI32, _PI32]),
    "kirin_get_launch": (ctypes.c_int, [_P, _I64, _PI32, _PI32]),
    "kirin_set_launch_table": (ctypes.c_int, [_P, _I32, _PI64, _PI32, _PI32]),
    "kirin_set_j_particles": (ctypes.c_int, [_P, _I64, _I64, _PD, _PD, _PD, _PD, _PD, _PD]),
    "kirin_set_j_particles_dev": (ctypes.c_int, [_P, _I64, _I64, _P, _P, _P, _P, _P, _P]),
    "kirin_set_nj": (ctypes.c_int, [_P, _I64]),
    "kirin_predict": (ctypes.c_int, [_P, _D]),
    "kirin_compute_forces": (ctypes.c_int, [_P, _I64, _PI32]),
    "kirin_get_acc_jerk_pot": (ctypes.c_int, [_P, _PD, _PD, _PD]),
    "kirin_compute_forces_dev": (ctypes.c_int, [_P, _I64, _P, _P, _P, _P]),
    "kirin_compute_forces_nn_dev": (ctypes.c_int, [_P, _I64, _P, _P, _P, _P, _P, _P]),
    "kirin_set_nn": (ctypes.c_int, [_P, _I32]),
    "kirin_get_nn": (ctypes.c_int, [_P, _PI32, _PD]),
    "kirin_sync": (ctypes.c_int, [_P]),
    "kirin_energy": (ctypes.c_int, [_P, _PD, _PD, _PD]),
    "kirin_hermite_init": (ctypes.c_int, [_P, _D, _D, _D, _D]),
    "kirin_hermite_block_step": (ctypes.c_int, [_P, _D, _PD, _PI64]),
    "kirin_hermite_run": (ctypes.c_int, [_P, _D, _I64, _PI64, _PD]),
    "kirin_set_device_loop": (ctypes.c_int, [_P, _I32]),
    "kirin_set_shared_persistent": (ctypes.c_int, [_P, _I32]),
    "kirin_get_shared_persistent": (ctypes.c_int, [_P, _PI32]),
    "kirin_set_tracing": (ctypes.c_int, [_P, _I32]),
    "kirin_get_trace": (ctypes.c_int, [_P, _PI64, _PD]),
    "kirin_hermite_shared_run": (ctypes.c_int, [_P, _D, _I64]),
    "kirin_hermite_shared_step": (ctypes.c_int, [_P, _D]),
    "kirin_get_state": (ctypes.c_int, [_P, _PD, _PD, _PD, _PD, _PD, _PD]),
    "kirin_set_state": (ctypes.c_int, [_P, _I64, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _D, _D, _D]),
    "kirin_selftest_wait_timeout": (ctypes.c_int, [_P, _I64]),
    "kirin_selftest_arrival_timeout": (ctypes.c_int, [_P, _I64]),
    "kirin_accel_dev": (ctypes.c_int, [_P, _I64, _P, _P, _P, _P]),
    "kirin_accel_adjoint_dev": (ctypes.c_int, [_P, _I64, _P, _P, _P, _P, _P]),
    "kirin_leapfrog_dev": (ctypes.c_int, [_P, _I64, _P, _P, _P, _P, _D, _I32, _I32, _P]),
    "kirin_leapfrog_adjoint_dev": (ctypes.c_int, [_P, _I64, _P, _P, _I32, _D, _P, _P, _P, _I32]),
    "kirin_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), _I32, _PI64, _PD, _D, _I32, _P]),
    "kirin_batch_destroy": (ctypes.c_int, [_P]),
    "kirin_batch_set_state": (ctypes.c_int, [_P, _PD, _PD, _PD]),
    "kirin_batch_get_state": (ctypes.c_int, [_P, _PD, _PD]),
    "kirin_batch_leapfrog": (ctypes.c_int, [_P, _D, _I32, _I32]),
    "kirin_batch_sync": (ctypes.c_int, [_P]),
    "kirin_batch_accel": (ctypes.c_int, [_P, _PD]),
    "kirin_batch_set_launch": (ctypes.c_int, [_P, _I32, _I32]),
    "kirin_batch_set_state_dev": (ctypes.c_int, [_P, _P, _P, _P]),
    "kirin_batch_get_state_dev": (ctypes.c_int, [_P, _P, _P]),
    "kirin_batch_accel_dev": (ctypes.c_int, [_P, _P]),
    "kirin_batch_get_launch": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "kirin_j_partition_range": (ctypes.c_int, [_I64, _I32, _I32, _PI64, _PI64]),
    "kirin_set_j_partition": (ctypes.c_int, [_P, _I32, _I32, _P, _P]),
    "kirin_forces_noalloc": (ctypes.c_int, [_I64, _P, _P, _P, _I64, _P, _D, _D, _D, _P, _P, _P, _P, _P]),
    "kirin_measure_fma_rate": (ctypes.c_int, [_I32, _I32, _PD]),
    "kirin_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "kirin_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None


def lib_path() -> str:
    """The in-tree libkirin.so, or the library named by $KIRIN_LIBRARY (a tuning variant)."""
    return os.environ.get("KIRIN_LIBRARY") or _build.LIB


def header_functions(path: str = HEADER):
    """Names of the functions declared in include/kirin.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kirin_\w+)\s*\(", text)))


def lib():
    """The loaded libkirin with argument types set (raises if it is not built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libkirin.so is not built ({path}); run __graft_entry__.build()")
        cdll = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(cdll, name)
            f.restype = res
            f.argtypes = args
        _lib = cdll
    return _lib


# kirin_allgather_fn: int (*)(void *user, const double *send, double *recv, int64_t count, void *stream)
ALLGATHER_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_void_p)


def j_partition_range(n_j: int, part: int, n_parts: int):
    """(j_begin, j_end): the j-particles part `part` of `n_parts` sums (kirin_j_partition_range)."""
    b, e = ctypes.c_int64(), ctypes.c_int64()
    rc = lib().kirin_j_partition_range(int(n_j), int(part), int(n_parts), ctypes.byref(b), ctypes.byref(e))
    if rc != KIRIN_OK:
        raise KirinError(rc, "kirin_j_partition_range")
    return b.value, e.value


def _strerror(code: int) -> str:
    try:
        return lib().kirin_strerror(code).decode()
    except Exception:  # the library itself may be what is missing
        return "?"


def _dp(a):
    return None if a is None else a.ctypes.data_as(_PD)


def _host(a, shape=None, dtype=np.float64):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream


def stream_handle(stream):
    """ctypes value of a stream argument: None lets the library create its own
    stream; 0 (the handle torch reports for its default stream) means the legacy
    default stream, passed as cudaStreamLegacy; anything else is a cudaStream_t."""
    if stream is None:
        return None
    stream = int(stream)
    return ctypes.c_void_p(CUDA_STREAM_LEGACY if stream == 0 else stream)


def _dev(t):
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Kirin:
    """One libkirin context (GPU_open ... GPU_close of Appendix A)."""

    def __init__(self, n_max, eps, G=1.0, r_min=0.0, precision="mixed", device=0, stream=None):
        self.lib = lib()
        cfg = kirin_config(float(eps), float(G), float(r_min), _prec(precision), int(device), stream_handle(stream))
        h = ctypes.c_void_p()
        self._check(self.lib.kirin_init(ctypes.byref(h), int(n_max), ctypes.byref(cfg)), "kirin_init", ctx=False)
        self.ctx = h
        self.n_max = int(n_max)
        self.n_j = 0
        self._pending = 0
        self.stream = stream

    def _check(self, rc, what, ctx=True):
        if rc != KIRIN_OK:
            detail = ""
            if ctx and getattr(self, "ctx", None):
                detail = self.lib.kirin_last_error(self.ctx).decode()
            box = getattr(self, "_exchange_box", None)
            if rc == KIRIN_EEXCHANGE and box and box[0] is not None:
                exc, box[0] = box[0], None
                raise KirinError(rc, what, detail) from exc
            raise KirinError(rc, what, detail)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.kirin_finalize(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- configuration
    def set_params(self, eps, G=1.0, r_min=0.0, precision="mixed"):
        self._check(self.lib.kirin_set_params(self.ctx, float(eps), float(G), float(r_min), _prec(precision)),
                    "kirin_set_params")

    def set_stream(self, stream):
        self._check(self.lib.kirin_set_stream(self.ctx, stream_handle(stream)), "kirin_set_stream")
        self.stream = stream

    def set_launch(self, groups=0, n_split=0):
        self._check(self.lib.kirin_set_launch(self.ctx, int(groups), int(n_split)), "kirin_set_launch")

    def set_launch_table(self, entries, kind=KIRIN_CALL_FORCES):
        """entries: [(n_i_max, groups, n_split), ...] ascending in n_i_max; [] clears the table.
        kind: which force calls it serves (KIRIN_CALL_FORCES, _ACC_POT or _ADJOINT)."""
        ni = np.ascontiguousarray([e[0] for e in entries], dtype=np.int64)
        gr = np.ascontiguousarray([e[1] for e in entries], dtype=np.int32)
        sp = np.ascontiguousarray([e[2] for e in entries], dtype=np.int32)
        self._check(self.lib.kirin_set_launch_table_for(self.ctx, int(kind), len(entries), ni.ctypes.data_as(_PI64),
                                                        gr.ctypes.data_as(_PI32), sp.ctypes.data_as(_PI32)),
                    "kirin_set_launch_table_for")

    def get_launch(self, n_i, kind=KIRIN_CALL_FORCES):
        g, s = ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.kirin_get_launch_for(self.ctx, int(kind), int(n_i), ctypes.byref(g), ctypes.byref(s)),
                    "kirin_get_launch_for")
        return g.value, s.value

    def query(self):
        n, ti, tj = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.kirin_query(self.ctx, ctypes.byref(n), ctypes.byref(ti), ctypes.byref(tj)),
                    "kirin_query")
        return n.value, ti.value, tj.value

    # -- GPU_set_j_particle / GPU_set_ti
    def set_j_particles(self, m, x, v, a=None, jerk=None, t0=None, first=0):
        m = _host(m)
        n = m.shape[0]
        x, v = _host(x, (n, 3)), _host(v, (n, 3))
        a, jerk, t0 = _host(a, (n, 3)), _host(jerk, (n, 3)), _host(t0, (n,))
        self._check(self.lib.kirin_set_j_particles(self.ctx, int(first), n, _dp(m), _dp(x), _dp(v), _dp(a),
                                                   _dp(jerk), _dp(t0)), "kirin_set_j_particles")
        self.n_j = max(self.n_j, first + n)

    def set_j_particles_dev(self, m, x, v, a=None, jerk=None, t0=None, first=0):
        n = m.shape[0]
        self._check(self.lib.kirin_set_j_particles_dev(self.ctx, int(first), int(n), _dev(m), _dev(x), _dev(v),
                                                       _dev(a), _dev(jerk), _dev(t0)), "kirin_set_j_particles_dev")
        self.n_j = max(self.n_j, first + n)

    def set_nj(self, n_j):
        self._check(self.lib.kirin_set_nj(self.ctx, int(n_j)), "kirin_set_nj")
        self.n_j = int(n_j)

    def predict(self, t):
        self._check(self.lib.kirin_predict(self.ctx, float(t)), "kirin_predict")

    # -- GPUcalc_firsthalf / GPUcalc_lasthalf
    def compute_forces(self, i_list=None):
        if i_list is None:
            self._check(self.lib.kirin_compute_forces(self.ctx, 0, None), "kirin_compute_forces")
            self._pending = self.n_j
        else:
            il = np.ascontiguousarray(i_list, dtype=np.int32)
            self._check(self.lib.kirin_compute_forces(self.ctx, il.shape[0], il.ctypes.data_as(_PI32)),
                        "kirin_compute_forces")
            self._pending = il.shape[0]

    def get_acc_jerk_pot(self):
        n = self._pending
        acc, jerk, pot = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
        self._check(self.lib.kirin_get_acc_jerk_pot(self.ctx, _dp(acc), _dp(jerk), _dp(pot)), "kirin_get_acc_jerk_pot")
        return acc, jerk, pot

    def forces(self, i_list=None):
        self.compute_forces(i_list)
        return self.get_acc_jerk_pot()

    def compute_forces_dev(self, i_list, acc, jerk, pot):
        """Device arrays (torch): i_list int32 (n_i) or None, acc/jerk (n_i, 3) and pot (n_i) float64.
        An empty i_list does nothing (the C call reads a NULL list, which an empty tensor has, as all j)."""
        if i_list is not None and i_list.numel() == 0:
            return
        n_i = self.n_j if i_list is None else i_list.shape[0]
        self._check(self.lib.kirin_compute_forces_dev(self.ctx, int(n_i), _dev(i_list), _dev(acc), _dev(jerk),
                                                      _dev(pot)), "kirin_compute_forces_dev")

    def compute_forces_nn_dev(self, i_list, acc, jerk, pot, nn, nn_r2):
        if i_list is not None and i_list.numel() == 0:
            return
        n_i = self.n_j if i_list is None else i_list.shape[0]
        self._check(self.lib.kirin_compute_forces_nn_dev(self.ctx, int(n_i), _dev(i_list), _dev(acc), _dev(jerk),
                                                         _dev(pot), _dev(nn), _dev(nn_r2)),
                    "kirin_compute_forces_nn_dev")

    def set_j_partition(self, part, n_parts, allgather=None):
        """Sum only part `part` of `n_parts` of the j tiles (kirin_set_j_partition).  allgather: None (results
        are this part's partial sums) or a callable (send, recv, count, stream) -> int over device pointers
        (ints), e.g. a jsplit.TorchAllGather; the context keeps it alive."""
        cb = None
        box = self._exchange_box = [None]  # the callback's failure, without a reference back to self
        if allgather is not None:
            def trampoline(user, send, recv, count, stream, _f=allgather, _box=box):
                try:
                    return int(_f(send, recv, count, stream))
                except BaseException as exc:  # never let ctypes swallow a failed exchange
                    _box[0] = exc
                    return 1
            cb = ALLGATHER_FN(trampoline)
        rc = self.lib.kirin_set_j_partition(self.ctx, int(part), int(n_parts),
                                            ctypes.cast(cb, ctypes.c_void_p) if cb is not None else None, None)
        self._check(rc, "kirin_set_j_partition")
        self._allgather_cb = cb  # the library holds the pointer: keep the thunk alive

    def set_nn(self, enable=True):
        self._check(self.lib.kirin_set_nn(self.ctx, 1 if enable else 0), "kirin_set_nn")

    def get_nn(self):
        n = self._pending
        nn = np.empty(n, dtype=np.int32)
        r2 = np.empty(n)
        self._check(self.lib.kirin_get_nn(self.ctx, nn.ctypes.data_as(_PI32), _dp(r2)), "kirin_get_nn")
        return nn, r2

    def sync(self):
        self._check(self.lib.kirin_sync(self.ctx), "kirin_sync")

    def energy(self, v=None):
        k, w = ctypes.c_double(), ctypes.c_double()
        vv = _host(v, (self.n_j, 3))
        self._check(self.lib.kirin_energy(self.ctx, _dp(vv), ctypes.byref(k), ctypes.byref(w)), "kirin_energy")
        return k.value, w.value

    # -- Hermite integrator
    def hermite_init(self, t=0.0, eta=0.01, dt_min=2.0 ** -20, dt_max=2.0 ** -3):
        self._check(self.lib.kirin_hermite_init(self.ctx, float(t), float(eta), float(dt_min), float(dt_max)),
                    "kirin_hermite_init")

    def hermite_block_step(self, t_end):
        t, n = ctypes.c_double(), ctypes.c_int64()
        self._check(self.lib.kirin_hermite_block_step(self.ctx, float(t_end), ctypes.byref(t), ctypes.byref(n)),
                    "kirin_hermite_block_step")
        return t.value, n.value

    def hermite_run(self, t_end, max_steps=0):
        """Block steps to t_end; returns (steps, pairs).  One graph launch per
        call unless set_device_loop(False)."""
        s, p = ctypes.c_int64(), ctypes.c_double()
        self._check(self.lib.kirin_hermite_run(self.ctx, float(t_end), int(max_steps), ctypes.byref(s),
                                               ctypes.byref(p)), "kirin_hermite_run")
        return s.value, p.value

    def set_device_loop(self, enable=True):
        self._check(self.lib.kirin_set_device_loop(self.ctx, 1 if enable else 0), "kirin_set_device_loop")

    def set_tracing(self, enable=True):
        """Time the device work of this context's compute calls with CUDA events (and name them in
        NVTX ranges); the totals start again from zero."""
        self._check(self.lib.kirin_set_tracing(self.ctx, 1 if enable else 0), "kirin_set_tracing")

    def get_trace(self):
        """(timed calls, their device time in ms) since the last set_tracing."""
        n, ms = ctypes.c_int64(), ctypes.c_double()
        self._check(self.lib.kirin_get_trace(self.ctx, ctypes.byref(n), ctypes.byref(ms)), "kirin_get_trace")
        return n.value, ms.value

    def set_shared_persistent(self, enable=True):
        """Let shared-step runs of small mixed-precision systems take the single-launch kernel."""
        self._check(self.lib.kirin_set_shared_persistent(self.ctx, 1 if enable else 0),
                    "kirin_set_shared_persistent")

    def shared_persistent_active(self):
        """Whether the next kirin_hermite_shared_run takes the single-launch kernel."""
        a = ctypes.c_int32()
        self._check(self.lib.kirin_get_shared_persistent(self.ctx, ctypes.byref(a)), "kirin_get_shared_persistent")
        return bool(a.value)

    def hermite_shared_step(self, dt):
        self._check(self.lib.kirin_hermite_shared_step(self.ctx, float(dt)), "kirin_hermite_shared_step")

    def hermite_shared_run(self, dt, n_steps):
        """n_steps shared steps, one synchronisation at the end."""
        self._check(self.lib.kirin_hermite_shared_run(self.ctx, float(dt), int(n_steps)), "kirin_hermite_shared_run")

    def get_state(self):
        n = self.n_j
        x, v, a, j = (np.empty((n, 3)) for _ in range(4))
        t, dt = np.empty(n), np.empty(n)
        self._check(self.lib.kirin_get_state(self.ctx, _dp(x), _dp(v), _dp(a), _dp(j), _dp(t), _dp(dt)),
                    "kirin_get_state")
        return {"x": x, "v": v, "a": a, "j": j, "t": t, "dt": dt}

    def set_state(self, m, st, eta=0.01, dt_min=2.0 ** -20, dt_max=2.0 ** -3):
        """Resume from a get_state() dictionary (plus the masses)."""
        m = _host(m)
        n = m.shape[0]
        arrs = [_host(st[k], (n, 3)) for k in ("x", "v", "a", "j")] + [_host(st["t"], (n,)), _host(st["dt"], (n,))]
        self._check(self.lib.kirin_set_state(self.ctx, n, _dp(m), *[_dp(a) for a in arrs], float(eta),
                                             float(dt_min), float(dt_max)), "kirin_set_state")
        self.n_j = n

    def selftest_wait_timeout(self, limit_ns=1_000_000):
        """Run the bounded-wait self-test; returns the library's return code (KIRIN_ETIMEOUT expected)."""
        return self.lib.kirin_selftest_wait_timeout(self.ctx, int(limit_ns))

    def selftest_arrival_timeout(self, limit_ns=1_000_000):
        """Device wait for an arrival that never comes: returns KIRIN_ETIMEOUT (not an exception)."""
        return self.lib.kirin_selftest_arrival_timeout(self.ctx, int(limit_ns))

    # -- device particle sets
    def accel_dev(self, m, x, acc, pot=None):
        self._check(self.lib.kirin_accel_dev(self.ctx, int(m.shape[0]), _dev(m), _dev(x), _dev(acc), _dev(pot)),
                    "kirin_accel_dev")

    def accel_adjoint_dev(self, m, x, g, gx, gm):
        self._check(self.lib.kirin_accel_adjoint_dev(self.ctx, int(m.shape[0]), _dev(m), _dev(x), _dev(g), _dev(gx),
                                                     _dev(gm)), "kirin_accel_adjoint_dev")

    def leapfrog_dev(self, m, x, v, acc, dt, n_steps, acc_valid=False, x_hist=None):
        self._check(self.lib.kirin_leapfrog_dev(self.ctx, int(m.shape[0]), _dev(m), _dev(x), _dev(v), _dev(acc),
                                                float(dt), int(n_steps), 1 if acc_valid else 0, _dev(x_hist)),
                    "kirin_leapfrog_dev")

    def leapfrog_adjoint_dev(self, m, x_hist, n_steps, dt, lx, lv, lm, flags):
        self._check(self.lib.kirin_leapfrog_adjoint_dev(self.ctx, int(m.shape[0]), _dev(m), _dev(x_hist),
                                                        int(n_steps), float(dt), _dev(lx), _dev(lv), _dev(lm),
                                                        int(flags)), "kirin_leapfrog_adjoint_dev")


class KirinBatch:
    """Many independent clusters advanced together (kirin_batch_*)."""

    def __init__(self, offsets, eps, G=1.0, device=0, stream=None):
        self.lib = lib()
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        ep = np.ascontiguousarray(eps, dtype=np.float64)
        h = ctypes.c_void_p()
        rc = self.lib.kirin_batch_create(ctypes.byref(h), off.shape[0] - 1, off.ctypes.data_as(_PI64), _dp(ep),
                                         float(G), int(device), stream_handle(stream))
        if rc != KIRIN_OK:
            raise KirinError(rc, "kirin_batch_create")
        self.b = h
        self.n_total = int(off[-1])

    def _check(self, rc, what):
        if rc != KIRIN_OK:
            raise KirinError(rc, what)

    def set_state(self, m, x, v):
        n = self.n_total
        m, x, v = _host(m, (n,)), _host(x, (n, 3)), _host(v, (n, 3))
        self._check(self.lib.kirin_batch_set_state(self.b, _dp(m), _dp(x), _dp(v)), "kirin_batch_set_state")

    def get_state(self):
        x, v = np.empty((self.n_total, 3)), np.empty((self.n_total, 3))
        self._check(self.lib.kirin_batch_get_state(self.b, _dp(x), _dp(v)), "kirin_batch_get_state")
        return x, v

    def leapfrog(self, dt, n_steps, use_graph=True):
        self._check(self.lib.kirin_batch_leapfrog(self.b, float(dt), int(n_steps), 1 if use_graph else 0),
                    "kirin_batch_leapfrog")

    def sync(self):
        self._check(self.lib.kirin_batch_sync(self.b), "kirin_batch_sync")

    def accel(self):
        acc = np.empty((self.n_total, 3))
        self._check(self.lib.kirin_batch_accel(self.b, _dp(acc)), "kirin_batch_accel")
        return acc

    def _dev_state(self, t, cols):
        """Device pointer of a contiguous CUDA float64 tensor of n_total (x cols) entries."""
        import torch
        shape = (self.n_total,) if cols == 1 else (self.n_total, cols)
        if t.dtype != torch.float64 or tuple(t.shape) != shape:
            raise ValueError(f"expected a float64 CUDA tensor of shape {shape}")
        return _dev(t)

    def set_state_dev(self, m, x, v):
        """State from CUDA tensors m (n_total,), x, v (n_total, 3); asynchronous on the batch's stream."""
        self._check(self.lib.kirin_batch_set_state_dev(self.b, self._dev_state(m, 1), self._dev_state(x, 3),
                                                       self._dev_state(v, 3)), "kirin_batch_set_state_dev")

    def get_state_dev(self, x=None, v=None):
        """Copy the positions and/or velocities into CUDA tensors (n_total, 3); asynchronous."""
        self._check(self.lib.kirin_batch_get_state_dev(self.b, None if x is None else self._dev_state(x, 3),
                                                       None if v is None else self._dev_state(v, 3)),
                    "kirin_batch_get_state_dev")

    def accel_dev(self, acc):
        """Accelerations into a CUDA tensor (n_total, 3); asynchronous."""
        self._check(self.lib.kirin_batch_accel_dev(self.b, self._dev_state(acc, 3)), "kirin_batch_accel_dev")

    def set_launch(self, groups, j_tiles):
        """Work items: blocks of 512 / groups i against at most j_tiles tiles of 128 j (0: whole clusters)."""
        self._check(self.lib.kirin_batch_set_launch(self.b, int(groups), int(j_tiles)), "kirin_batch_set_launch")

    def get_launch(self):
        """(groups, j_tiles, number of work items)."""
        g, jt, ni = _I32(), _I32(), _I32()
        self._check(self.lib.kirin_batch_get_launch(self.b, ctypes.byref(g), ctypes.byref(jt), ctypes.byref(ni)),
                    "kirin_batch_get_launch")
        return g.value, jt.value, ni.value

    def close(self):
        if getattr(self, "b", None):
            self.lib.kirin_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_fma_rate(kind: str, device: int = 0) -> float:
    """Measured FMA throughput in flop/s: kind "fp32", "fp32x2" or "fp64"."""
    code = {"fp32": 0, "fp32x2": 1, "fp64": 2}[kind]
    out = ctypes.c_double()
    rc = lib().kirin_measure_fma_rate(int(device), code, ctypes.byref(out))
    if rc != KIRIN_OK:
        raise KirinError(rc, "kirin_measure_fma_rate")
    return out.value


def _prec(p) -> int:
    if p in ("mixed", KIRIN_MIXED):
        return KIRIN_MIXED
    if p in ("fp64", KIRIN_FP64):
        return KIRIN_FP64
    raise ValueError(f"unknown precision {p!r}")
