"""The device-driven block-step loop of kirin_hermite_run (one CUDA graph with a
conditional WHILE node and a SWITCH over force launches) against the same steps
taken with one host round trip each (Sect. 3.1 block time-steps), and against
the oracle's schedule."""
import numpy as np
import pytest

from oracle import hermite
from paper_0707_0438_gb300 import abi, metrics, workloads

pytestmark = pytest.mark.gpu

STATE_KEYS = ("x", "v", "a", "j", "t", "dt")
FIXED = {"mixed": (2, 4), "fp64": (1, 4)}


def _run(p, precision, device_loop, t_ends, launch=None, max_steps=0):
    """Block steps to each t_end in turn; returns [(steps, pairs)], the state and the energy."""
    with abi.Kirin(p.n, p.eps, precision=precision) as k:
        if launch:
            k.set_launch(*launch)
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(0.0)
        k.set_device_loop(device_loop)
        counts = [k.hermite_run(t, max_steps) for t in t_ends]
        st = k.get_state()
        e = sum(k.energy())
    return counts, st, e


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("n", [4096, 48])
def test_device_loop_is_bitwise_the_host_loop(kirin_lib, precision, n):
    """Same fixed launch shape: identical step counts, pair counts and state, over
    two calls with different end times (one graph, t_end read on the device)."""
    p = workloads.plummer(n, 1002, eps=1e-3)
    t_ends = [1.0 / 64, 1.0 / 32]
    host = _run(p, precision, False, t_ends, FIXED[precision])
    dev = _run(p, precision, True, t_ends, FIXED[precision])
    assert dev[0] == host[0]
    assert all(c[0] > 0 for c in dev[0])
    for key in STATE_KEYS:
        assert np.array_equal(dev[1][key], host[1][key]), key
    assert dev[2] == host[2]


@pytest.mark.parametrize("n,t_end", [(256, 1.0 / 8), (4096, 1.0 / 8), (8192, 1.0 / 32)])
def test_device_loop_fp64_follows_the_oracle_schedule(kirin_lib, n, t_end):
    """Automatic shapes (a ladder of launches by block size): the oracle's block
    sequence length and pair count, its times and steps exactly, its positions
    to FP64 rounding.  N = 4096 to t = 1/8 takes 1300 block steps, N = 8192 to
    1/32 621, with blocks from one particle to all of them."""
    p = workloads.plummer(n, 1002, eps=1e-3)
    ref = hermite.block_steps(p.m, p.x, p.v, p.eps, t_end=t_end)
    [(steps, pairs)], st, e = _run(p, "fp64", True, [t_end])
    assert steps == len(ref["blocks"])
    assert pairs == float(sum(ref["blocks"])) * p.n
    assert np.array_equal(st["t"], ref["t"])
    assert np.array_equal(st["dt"], ref["dt"])
    assert np.abs(st["x"] - ref["x"]).max() <= 1e-9
    if t_end % hermite.DT_MAX == 0:  # a multiple of the largest step: every particle ends there, and
        assert np.all(st["t"] == t_end)  # the energy of the synchronised state is defined
        assert e == pytest.approx(ref["e_end"], rel=1e-10)


def test_device_loop_max_steps_and_rebuild_on_new_shape(kirin_lib):
    """max_steps stops the device loop exactly; a later call resumes it; changing
    the launch shape between calls rebuilds the graph (results stay those of the
    host loop under the same shapes)."""
    p = workloads.plummer(2048, 1005, eps=1e-3)
    t_end = 1.0 / 32
    with abi.Kirin(p.n, p.eps, precision="mixed") as kd, abi.Kirin(p.n, p.eps, precision="mixed") as kh:
        for k, dev in ((kd, True), (kh, False)):
            k.set_launch(2, 4)
            k.set_j_particles(p.m, p.x, p.v)
            k.hermite_init(0.0)
            k.set_device_loop(dev)
        a = kd.hermite_run(t_end, 5)
        b = kh.hermite_run(t_end, 5)
        assert a == b and a[0] == 5
        for k in (kd, kh):
            k.set_launch(4, 8)
        a = kd.hermite_run(t_end)
        b = kh.hermite_run(t_end)
        assert a == b and a[0] > 0
        sd, sh = kd.get_state(), kh.get_state()
        assert kd.hermite_run(t_end) == (0, 0.0)  # nothing left before t_end
    for key in STATE_KEYS:
        assert np.array_equal(sd[key], sh[key]), key
    # every particle stepped as far as it can without passing t_end
    assert np.all(sd["t"] <= t_end) and np.all(sd["t"] + sd["dt"] > t_end)


def test_device_loop_automatic_shapes_mixed(kirin_lib):
    """Mixed precision with automatic shapes on both paths (the device ladder and
    the host's per-block choice differ in summation order only): the same energy
    to the mixed kernel's rounding, positions to 1e-9 of their scale."""
    p = workloads.plummer(16384, 1002, eps=1e-3)
    t_end = 1.0 / 64
    host = _run(p, "mixed", False, [t_end])
    dev = _run(p, "mixed", True, [t_end])
    (sh, ph), (sd, pd) = host[0][0], dev[0][0]
    assert abs(sd - sh) <= 2 and sd > 0
    t, dt = dev[1]["t"], dev[1]["dt"]
    assert np.all(t <= t_end) and np.all(t + dt > t_end)
    scale = np.abs(p.x).max()
    assert np.abs(dev[1]["x"] - host[1]["x"]).max() <= 1e-9 * scale
    assert dev[2] == pytest.approx(host[2], rel=1e-9)


@pytest.mark.parametrize("device_loop", [True, False])
def test_block_time_that_stops_advancing_is_an_error(kirin_lib, device_loop):
    """At t = 2^60 a step of 2^-20 rounds away (t + dt == t in FP64): both loops stop
    with an error instead of repeating the same block forever."""
    p = workloads.plummer(256, 1002, eps=1e-3)
    with abi.Kirin(p.n, p.eps, precision="fp64") as k:
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(0.0)
        st = k.get_state()
        st["t"][:] = 2.0 ** 60
        st["dt"][:] = 2.0 ** -20
        k.set_state(p.m, st, dt_min=2.0 ** -20, dt_max=2.0 ** -3)
        k.set_device_loop(device_loop)
        with pytest.raises(abi.KirinError):
            k.hermite_run(2.0 ** 60 + 2.0 ** 10)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("n,eps,r_min", [(1, 1e-2, 0.0), (2, 1e-2, 0.0), (129, 0.0, 1e-6)])
def test_device_loop_edge_sizes(kirin_lib, precision, n, eps, r_min):
    """One particle (no force, no jerk: the step criterion is 0/0 and the step is kept), a pair, and a
    ragged 129 with eps = 0 and the r_min guard: the device loop matches the host loop bit for bit under a
    fixed launch shape, and keeps its schedule with the automatic shapes (tiny-block kernel included)."""
    p = workloads.plummer(n, (1006, n), eps=eps)

    def run(device_loop, launch):
        with abi.Kirin(p.n, eps, r_min=r_min, precision=precision) as k:
            if launch:
                k.set_launch(*launch)
            k.set_j_particles(p.m, p.x, p.v)
            k.hermite_init(0.0)
            k.set_device_loop(device_loop)
            counts = k.hermite_run(1.0 / 8)  # = dt_max: a lone particle (dt = dt_max) steps once
            return counts, k.get_state()

    host = run(False, (1, 2))
    dev = run(True, (1, 2))
    assert dev[0] == host[0] and dev[0][0] > 0
    for key in STATE_KEYS:
        assert np.array_equal(dev[1][key], host[1][key]), key
    auto_h, auto_d = run(False, None), run(True, None)
    assert auto_d[0][0] == auto_h[0][0]
    assert np.array_equal(auto_d[1]["t"], auto_h[1]["t"]) and np.array_equal(auto_d[1]["dt"], auto_h[1]["dt"])
    assert np.allclose(auto_d[1]["x"], auto_h[1]["x"], rtol=0, atol=1e-9 * max(1.0, np.abs(p.x).max()))
    assert np.all(np.isfinite(auto_d[1]["x"]))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_device_loop_with_one_level_is_the_shared_run(kirin_lib, precision):
    """dt_min = dt_max: every block is every particle, so the device-driven block loop must reproduce
    kirin_hermite_shared_run bit for bit under one launch shape (two independent paths: the step
    kernels' selection, prediction and correction against the predictor/corrector kernels)."""
    p = workloads.plummer(3000, 1007, eps=1e-3)
    dt = 2.0 ** -8
    out = []
    for shared in (True, False):
        with abi.Kirin(p.n, p.eps, precision=precision) as k:
            k.set_launch(2, 4)
            k.set_j_particles(p.m, p.x, p.v)
            k.hermite_init(0.0, dt_min=dt, dt_max=dt)
            if shared:
                k.hermite_shared_run(dt, 16)
            else:
                steps, pairs = k.hermite_run(16 * dt)
                assert steps == 16 and pairs == 16.0 * p.n * p.n
            out.append(k.get_state())
    for key in ("x", "v", "a", "j", "t", "dt"):
        assert np.array_equal(out[0][key], out[1][key]), key


def test_device_loop_long_run(kirin_lib):
    """Thousands of block steps in one graph launch (N = 2048 to t = 1/2, four dt_max periods): energy
    conserved, every particle synchronised at t_end, the host loop's step count, and a second call
    that continues from there."""
    p = workloads.plummer(2048, 1008, eps=1e-3)
    counts = {}
    for device_loop in (True, False):
        with abi.Kirin(p.n, p.eps, precision="mixed") as k:
            k.set_j_particles(p.m, p.x, p.v)
            e0 = sum(k.energy())
            k.hermite_init(0.0)
            k.set_device_loop(device_loop)
            steps, _ = k.hermite_run(0.5)
            st = k.get_state()
            e1 = sum(k.energy())
            more, _ = k.hermite_run(0.625)
            counts[device_loop] = (steps, more)
        assert np.all(st["t"] == 0.5)
        assert abs(metrics.energy_error(e0, e1)) < 1e-5
    assert counts[True][0] > 1000 and counts[True][1] > 0
    assert abs(counts[True][0] - counts[False][0]) <= 0.01 * counts[False][0]


@pytest.mark.parametrize("device_loop", [True, False])
def test_block_steps_from_a_negative_time(kirin_lib, device_loop):
    """Block times are ordered as numbers, not as bit patterns: a run that starts at t = -1/8 reaches
    t = 0 exactly as a run shifted to start at 0 reaches 1/8 (same schedule, same state)."""
    p = workloads.plummer(1024, 1009, eps=1e-3)
    results = []
    for t0 in (-0.125, 0.0):
        with abi.Kirin(p.n, p.eps, precision="mixed") as k:
            k.set_launch(2, 4)
            k.set_j_particles(p.m, p.x, p.v)
            k.hermite_init(t0)
            k.set_device_loop(device_loop)
            steps, pairs = k.hermite_run(t0 + 0.125)
            st = k.get_state()
        assert np.all(st["t"] == t0 + 0.125)
        results.append((steps, st))
    assert results[0][0] == results[1][0] > 0
    for key in ("x", "v", "a", "j", "dt"):
        assert np.array_equal(results[0][1][key], results[1][1][key]), key


def test_host_and_device_steps_interleave(kirin_lib):
    """Host-driven block steps, then a device-driven run limited by max_steps, then host steps to the end
    reproduce a pure host-driven run bit for bit (one launch shape): each driver leaves a state the other
    continues from."""
    p = workloads.plummer(2048, 1010, eps=1e-3)
    t_end = 1.0 / 16

    def ctx():
        k = abi.Kirin(p.n, p.eps, precision="mixed")
        k.set_launch(4, 4)
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(0.0)
        return k

    with ctx() as k:
        k.set_device_loop(False)
        total, _ = k.hermite_run(t_end)
        ref = k.get_state()
    with ctx() as k:
        done = 0
        for _ in range(7):
            _, n_act = k.hermite_block_step(t_end)
            done += n_act > 0
        k.set_device_loop(True)
        steps, _ = k.hermite_run(t_end, 50)
        done += steps
        while True:
            _, n_act = k.hermite_block_step(t_end)
            if n_act == 0:
                break
            done += 1
        st = k.get_state()
    assert done == total and steps == 50
    for key in STATE_KEYS:
        assert np.array_equal(st[key], ref[key]), key
