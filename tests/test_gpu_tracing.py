"""Tracing of a context's compute calls (kirin_set_tracing / kirin_get_trace): CUDA events around the
stream work of each traced call, NVTX ranges named after the calls.  Not in the paper, which times its
kernels with host timers and leaves transfers out (Sect. 4.1).  Checked here: the count of timed calls,
nested calls timed once, device time within the wall time, results bit for bit those of an untraced
context, and the totals reset by kirin_set_tracing."""
import time

import numpy as np
import pytest
import torch

from paper_0707_0438_gb300 import abi, workloads

pytestmark = pytest.mark.gpu


def test_tracing_counts_calls_and_device_time(kirin_lib):
    p = workloads.plummer(4096, 1021, eps=1e-2)
    with abi.Kirin(p.n, p.eps) as k:
        k.set_j_particles(p.m, p.x, p.v)
        ref = k.forces()
        assert k.get_trace() == (0, 0.0)  # off by default
        k.set_tracing(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs = [k.forces() for _ in range(3)]
        wall_ms = 1e3 * (time.perf_counter() - t0)
        n, ms = k.get_trace()
        assert n == 3
        assert 0.0 < ms <= wall_ms
        for out in outs:
            for a, b in zip(out, ref):
                np.testing.assert_array_equal(a, b)
        # a whole Hermite run is one timed call (the device loop, or the host loop's nested steps)
        k.hermite_init(0.0)
        k.hermite_run(1.0 / 64)
        n2, ms2 = k.get_trace()
        assert n2 == 5 and ms2 > ms
        k.set_device_loop(False)
        k.hermite_run(2.0 / 64)
        assert k.get_trace()[0] == 6
        k.set_tracing(False)
        k.forces()
        assert k.get_trace() == (0, 0.0)


def test_tracing_over_many_calls_folds_and_keeps_counting(kirin_lib):
    """More than 1024 timed calls: the pending event pairs are folded on the way, none is lost."""
    p = workloads.plummer(256, 1022, eps=1e-2)
    with abi.Kirin(p.n, p.eps) as k:
        k.set_j_particles(p.m, p.x, p.v)
        acc = torch.empty((p.n, 3), dtype=torch.float64, device="cuda")
        jerk = torch.empty_like(acc)
        pot = torch.empty(p.n, dtype=torch.float64, device="cuda")
        k.set_tracing(True)
        for _ in range(1500):
            k.compute_forces_dev(None, acc, jerk, pot)
        n, ms = k.get_trace()
        assert n == 1500 and ms > 0.0
