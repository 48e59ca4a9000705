"""kirin_forces_noalloc: the allocation-free variant of the mixed-precision force
evaluation, for callers that cannot allocate device memory when they need forces
(inside another framework's memory pool, or where cudaMalloc would synchronise the
device).  It must give the results of the context path (kirin_compute_forces_dev)
and of the FP64 oracle within the tests' mixed-precision tolerance, call after call,
although every call reuses the same static scratch, and it must leave the device's
free memory unchanged.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0707_0438_gb300 import abi, workloads
from tests.gpu_util import assert_parity

pytestmark = pytest.mark.gpu


def _case(n, seed, n_i, eps=1.0 / 256):
    import torch
    dev = torch.device("cuda:0")
    p = workloads.plummer(n, seed, masses="lognormal", eps=eps)
    t = tuple(torch.tensor(a, device=dev) for a in (p.m, p.x, p.v))
    il = torch.tensor(workloads.i_subset(n, n_i, seed), device=dev)
    return p, t, il


def _outputs(n_i, fill=np.nan):
    import torch
    dev = torch.device("cuda:0")
    return tuple(torch.full(s, fill, dtype=torch.float64, device=dev) for s in ((n_i, 3), (n_i, 3), (n_i,)))


def _noalloc(t, n, il, n_i, eps, r_min, out, status, stream):
    return abi.lib().kirin_forces_noalloc(n, abi._dev(t[0]), abi._dev(t[1]), abi._dev(t[2]), n_i, abi._dev(il),
                                          eps, 1.0, r_min, abi._dev(out[0]), abi._dev(out[1]), abi._dev(out[2]),
                                          abi._dev(status), abi.stream_handle(stream))


def _context(t, n, il, eps, r_min, like, stream):
    import torch
    ref = tuple(torch.empty_like(o) for o in like)
    with abi.Kirin(n, eps, r_min=r_min, precision="mixed", stream=stream) as k:
        k.set_j_particles_dev(*t)
        k.compute_forces_dev(il, *ref)
        k.sync()
    return tuple(r.cpu().numpy() for r in ref)


def test_noalloc_matches_context_path_and_oracle_on_consecutive_calls(kirin_lib):
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row with different sizes: the second must not see the first's scratch
    for n, seed, n_i in ((20000, 11, 20000), (3000, 12, 700)):
        p, t, il = _case(n, seed, n_i)
        out = _outputs(n_i)
        status = torch.full((1,), 0xFFFF, dtype=torch.int32, device=dev)
        assert _noalloc(t, n, il, n_i, p.eps, 0.0, out, status, stream) == abi.KIRIN_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got = tuple(o.cpu().numpy() for o in out)
        assert_parity(got, _context(t, n, il, p.eps, 0.0, out, stream), "mixed", f"noalloc vs context n={n}")
        ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il.cpu().numpy())
        assert_parity(got, ref, "mixed", f"noalloc vs oracle n={n}")


def test_noalloc_zero_softening_guard_against_oracle(kirin_lib):
    """eps = 0 with the r_min = 1e-6 floor (Sect. 3.3.1) runs the guarded kernel, which has its own
    templates and occupancy; with a coincident distinct pair planted, and no status word (the scratch
    keeps its own)."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    n, n_i = 4099, 4099
    p = workloads.plummer(n, 14, masses="lognormal", eps=0.0)
    p.x[7] = p.x[3]  # a distinct particle at the same place: contributes nothing
    dev = torch.device("cuda:0")
    t = tuple(torch.tensor(a, device=dev) for a in (p.m, p.x, p.v))
    out = _outputs(n_i)
    assert _noalloc(t, n, None, n_i, 0.0, 1e-6, out, None, stream) == abi.KIRIN_OK
    torch.cuda.synchronize()
    got = tuple(o.cpu().numpy() for o in out)
    assert_parity(got, oracle.acc_jerk_pot(p.m, p.x, p.v, 0.0, r_min=1e-6), "mixed", "noalloc guard vs oracle")
    assert_parity(got, _context(t, n, None, 0.0, 1e-6, out, stream), "mixed", "noalloc guard vs context")


def test_noalloc_all_particles_and_status_words(kirin_lib):
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    p, t, _ = _case(5000, 13, 1)
    out = _outputs(5000)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    assert _noalloc(t, 5000, None, 0, p.eps, 0.0, out, status, stream) == abi.KIRIN_OK
    got = tuple(o.cpu().numpy() for o in out)
    assert_parity(got, _context(t, 5000, None, p.eps, 0.0, out, stream), "mixed")
    assert_parity(got, oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps), "mixed")
    # an index outside [0, n) is reported in the status word, not by a fault
    bad = torch.tensor([0, 5000, 3], dtype=torch.int32, device=dev)
    small = _outputs(3)
    assert _noalloc(t, 5000, bad, 3, p.eps, 0.0, small, status, stream) == abi.KIRIN_OK
    torch.cuda.synchronize()
    assert int(status.item()) & 1
    # a NaN in the input sets the non-finite bit, and the next clean call clears the word
    x_nan = t[1].clone()
    x_nan[11, 1] = float("nan")
    assert _noalloc((t[0], x_nan, t[2]), 5000, None, 0, p.eps, 0.0, out, status, stream) == abi.KIRIN_OK
    torch.cuda.synchronize()
    assert int(status.item()) & 8
    assert _noalloc(t, 5000, None, 0, p.eps, 0.0, out, status, stream) == abi.KIRIN_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0


def test_noalloc_leaves_free_device_memory_unchanged(kirin_lib):
    """The property the entry point exists for: once every launch shape it will use has run once,
    further calls of several sizes change the device's free memory (cudaMemGetInfo) by nothing."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    cases = []
    for n, n_i, eps, r_min in ((32768, 32768, 1e-3, 0.0), (5000, 37, 1e-3, 0.0), (1000, 1000, 0.0, 1e-6),
                               (20000, 900, 1.0 / 256, 0.0)):
        p, t, il = _case(n, 15, n_i, eps=eps)
        cases.append((t, n, il, n_i, eps, r_min, _outputs(n_i), torch.zeros(1, dtype=torch.int32, device="cuda")))

    def run_all():
        for c in cases:
            assert _noalloc(*c, stream) == abi.KIRIN_OK
        torch.cuda.synchronize()

    run_all()  # first use loads the kernels these shapes need
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        run_all()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for c in cases:
        assert int(c[-1].item()) == 0


def test_noalloc_rejects_sizes_beyond_its_scratch(kirin_lib):
    lib = abi.lib()
    n = 32769  # KIRIN_NOALLOC_MAX_N + 1; rejected before any device work
    assert lib.kirin_forces_noalloc(n, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), 0, None, 0.01,
                                    1.0, 0.0, None, None, None, None, None) == abi.KIRIN_EINVAL
    assert lib.kirin_forces_noalloc(100, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), 40000,
                                    ctypes.c_void_p(8), 0.01, 1.0, 0.0, None, None, None, None,
                                    None) == abi.KIRIN_EINVAL
