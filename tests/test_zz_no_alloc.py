"""kirin_forces_noalloc: the allocation-free variant of the mixed-precision force
evaluation, for callers that cannot allocate device memory when they need forces
(inside another framework's memory pool, or where cudaMalloc would synchronise the
device).  It must give the results of the context path (kirin_compute_forces_dev)
within the tests' mixed-precision tolerance, call after call, although every call
reuses the same static scratch.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_0707_0438_gb300 import abi, workloads
from tests.gpu_util import assert_parity

pytestmark = pytest.mark.gpu


def _case(n, seed, n_i):
    import torch
    dev = torch.device("cuda:0")
    p = workloads.plummer(n, seed, masses="lognormal", eps=1.0 / 256)
    t = tuple(torch.tensor(a, device=dev) for a in (p.m, p.x, p.v))
    il = torch.tensor(workloads.i_subset(n, n_i, seed), device=dev)
    return p, t, il


def test_noalloc_matches_context_path_on_consecutive_calls(kirin_lib):
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    lib = abi.lib()
    # two calls in a row with different sizes: the second must not see the first's scratch
    for n, seed, n_i in ((20000, 11, 20000), (3000, 12, 700)):
        p, t, il = _case(n, seed, n_i)
        out = tuple(torch.full(s, np.nan, dtype=torch.float64, device=dev) for s in ((n_i, 3), (n_i, 3), (n_i,)))
        status = torch.full((1,), 0xFFFF, dtype=torch.int32, device=dev)
        rc = lib.kirin_forces_noalloc(n, abi._dev(t[0]), abi._dev(t[1]), abi._dev(t[2]), n_i, abi._dev(il),
                                      p.eps, 1.0, 0.0, abi._dev(out[0]), abi._dev(out[1]), abi._dev(out[2]),
                                      abi._dev(status), abi.stream_handle(stream))
        assert rc == abi.KIRIN_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        ref = tuple(torch.empty_like(o) for o in out)
        with abi.Kirin(n, p.eps, precision="mixed", stream=stream) as k:
            k.set_j_particles_dev(*t)
            k.compute_forces_dev(il, *ref)
            k.sync()
        got = tuple(o.cpu().numpy() for o in out)
        assert_parity(got, tuple(r.cpu().numpy() for r in ref), "mixed", f"noalloc n={n}")


def test_noalloc_all_particles_and_status_words(kirin_lib):
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    lib = abi.lib()
    p, t, _ = _case(5000, 13, 1)
    out = tuple(torch.empty(s, dtype=torch.float64, device=dev) for s in ((5000, 3), (5000, 3), (5000,)))
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    assert lib.kirin_forces_noalloc(5000, abi._dev(t[0]), abi._dev(t[1]), abi._dev(t[2]), 0, None, p.eps, 1.0, 0.0,
                                    abi._dev(out[0]), abi._dev(out[1]), abi._dev(out[2]), abi._dev(status),
                                    abi.stream_handle(stream)) == abi.KIRIN_OK
    ref = tuple(torch.empty_like(o) for o in out)
    with abi.Kirin(5000, p.eps, precision="mixed", stream=stream) as k:
        k.set_j_particles_dev(*t)
        k.compute_forces_dev(None, *ref)
        k.sync()
    assert_parity(tuple(o.cpu().numpy() for o in out), tuple(r.cpu().numpy() for r in ref), "mixed")
    # an index outside [0, n) is reported in the status word, not by a fault
    bad = torch.tensor([0, 5000, 3], dtype=torch.int32, device=dev)
    small = tuple(torch.empty(s, dtype=torch.float64, device=dev) for s in ((3, 3), (3, 3), (3,)))
    assert lib.kirin_forces_noalloc(5000, abi._dev(t[0]), abi._dev(t[1]), abi._dev(t[2]), 3, abi._dev(bad), p.eps,
                                    1.0, 0.0, abi._dev(small[0]), abi._dev(small[1]), abi._dev(small[2]),
                                    abi._dev(status), abi.stream_handle(stream)) == abi.KIRIN_OK
    torch.cuda.synchronize()
    assert int(status.item()) & 1


def test_noalloc_rejects_sizes_beyond_its_scratch(kirin_lib):
    lib = abi.lib()
    n = 32769  # KIRIN_NOALLOC_MAX_N + 1; rejected before any device work
    assert lib.kirin_forces_noalloc(n, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), 0, None, 0.01,
                                    1.0, 0.0, None, None, None, None, None) == abi.KIRIN_EINVAL
    assert lib.kirin_forces_noalloc(100, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), 40000,
                                    ctypes.c_void_p(8), 0.01, 1.0, 0.0, None, None, None, None,
                                    None) == abi.KIRIN_EINVAL
