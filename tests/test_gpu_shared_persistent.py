"""Shared-step Hermite runs of small systems in one cooperative launch (one CTA per SM; the predicted
j image published through global memory and a grid barrier per step): against the FP64 oracle's
Hermite steps (Sect. 3) and against the per-kernel path, for ragged sizes up to 2048, with and without
the zero-softening guard."""
import numpy as np
import pytest

import oracle
from oracle import hermite
from paper_0707_0438_gb300 import abi, metrics, workloads

pytestmark = pytest.mark.gpu


def _run(p, eps, dt, steps, persistent, r_min=0.0):
    with abi.Kirin(p.n, eps, r_min=r_min, precision="mixed") as k:
        k.set_shared_persistent(persistent)
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(0.0)
        active = k.shared_persistent_active()
        k.hermite_shared_run(dt, steps)
        st = k.get_state()
        after = k.forces()  # the run leaves a consistent context behind
    return active, st, after


@pytest.mark.parametrize("n", [1, 2, 17, 151, 152, 153, 777, 1024, 1500, 2048])
def test_persistent_shared_run_matches_the_oracle(kirin_lib, n):
    """Sizes below, at and above one particle per CTA (152 SMs), ragged tiles and the largest system."""
    p = workloads.plummer(n, (1001, n), eps=1.0 / 256)
    dt, steps = 1.0 / 1024, 10
    xr, vr, ar, _, _ = hermite.shared_steps(p.m, p.x, p.v, p.eps, dt, steps)
    active, st, after = _run(p, p.eps, dt, steps, True)
    assert active
    assert np.all(st["t"] == steps * dt)
    assert np.abs(st["x"] - xr).max() <= 1e-7 * max(np.abs(p.x).max(), 1e-300)
    assert np.abs(st["v"] - vr).max() <= 1e-6 * max(np.abs(p.v).max(), 1e-300)
    if n > 1:
        assert np.median(metrics.rel_err_vec(st["a"], ar)) <= 1e-6
        ref = oracle.acc_jerk_pot(p.m, st["x"], st["v"], p.eps)
        assert np.median(metrics.rel_err_vec(after[0], ref[0])) <= 1e-6


@pytest.mark.parametrize("n", [2, 777, 2048])
def test_persistent_hermite_init_matches_the_oracle(kirin_lib, n):
    """kirin_hermite_init in one launch of the shared-step kernel: the first a and jerk against the
    oracle's, x and v untouched, t_i = t, and the initial steps 0.01 |a| / |jerk| on the power-of-two ladder
    (the oracle's quantiser applied to the oracle's forces; a force error of 1e-6 can only move a
    particle whose raw step sits that close to a power of two)."""
    p = workloads.plummer(n, (2002, n), eps=1.0 / 256)
    with abi.Kirin(p.n, p.eps, precision="mixed") as k:
        k.set_j_particles(p.m, p.x, p.v)
        assert k.shared_persistent_active()
        k.hermite_init(0.25)
        st = k.get_state()
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps)
    for got, want in ((st["a"], ref[0]), (st["j"], ref[1])):
        err = metrics.rel_err_vec(got, want)
        assert np.median(err) <= 1e-6 and err.max() <= 1e-4
    assert np.array_equal(st["x"], p.x) and np.array_equal(st["v"], p.v)
    assert np.all(st["t"] == 0.25)
    raw = 0.01 * np.linalg.norm(ref[0], axis=1) / np.linalg.norm(ref[1], axis=1)
    want_dt = hermite.quantise_initial(raw)
    near = np.abs(np.log2(raw) - np.round(np.log2(raw))) < 1e-5
    assert np.array_equal(st["dt"][~near], want_dt[~near])
    assert np.all(np.isin(st["dt"], [want_dt.min() / 2] + list(np.unique(want_dt)) + [want_dt.max() * 2]))


@pytest.mark.parametrize("n,eps,r_min,tol", [(1024, 1.0 / 256, 0.0, 1e-10), (900, 0.0, 1e-6, 1e-8)])
def test_persistent_shared_run_agrees_with_the_kernel_path(kirin_lib, n, eps, r_min, tol):
    """The same 64 steps through the single launch and through the predictor, force and corrector
    kernels.  The j are summed in other orders, so the states agree to rounding.  Without softening a
    close pair magnifies that difference step by step (3e-10 of max |x| measured after 64 steps),
    hence the wider bound there."""
    p = workloads.plummer(n, 4040, eps=eps)
    dt, steps = 1.0 / 1024, 64
    a_on, on, _ = _run(p, eps, dt, steps, True, r_min)
    a_off, off, _ = _run(p, eps, dt, steps, False, r_min)
    assert a_on and not a_off
    assert np.all(on["t"] == off["t"])
    assert np.abs(on["x"] - off["x"]).max() <= tol * np.abs(p.x).max()
    assert np.median(metrics.rel_err_vec(on["a"], off["a"])) <= 1e-6


def test_persistent_shared_run_is_deterministic(kirin_lib):
    """Two contexts, the same run: the same bits (fixed CTA slices, fixed reduction order)."""
    p = workloads.plummer(1500, 77, eps=1.0 / 256)
    _, a, fa = _run(p, p.eps, 1.0 / 1024, 20, True)
    _, b, fb = _run(p, p.eps, 1.0 / 1024, 20, True)
    for key in ("x", "v", "a", "j", "t", "dt"):
        assert np.array_equal(a[key], b[key]), key
    for u, w in zip(fa, fb):
        assert np.array_equal(u, w)


def test_persistent_shared_run_limits(kirin_lib):
    """Above 8192 particles, in FP64 and under a fixed launch shape the per-kernel path runs; a run of
    no steps changes nothing."""
    p = workloads.plummer(8193, 1, eps=0.01)
    with abi.Kirin(p.n, p.eps, precision="mixed") as k:
        k.set_j_particles(p.m, p.x, p.v)
        assert not k.shared_persistent_active()
    q = workloads.plummer(1000, 2, eps=0.01)
    with abi.Kirin(q.n, q.eps, precision="fp64") as k:
        k.set_j_particles(q.m, q.x, q.v)
        assert not k.shared_persistent_active()
    with abi.Kirin(q.n, q.eps, precision="mixed") as k:
        k.set_j_particles(q.m, q.x, q.v)
        assert k.shared_persistent_active()
        k.hermite_init(0.0)
        before = k.get_state()
        k.hermite_shared_run(1.0 / 1024, 0)  # no steps: nothing changes
        after = k.get_state()
        for key in ("x", "v", "a", "j", "t", "dt"):
            assert np.array_equal(before[key], after[key]), key
        k.set_launch(2, 4)
        assert not k.shared_persistent_active()


def test_persistent_shared_run_guard_with_a_coincident_pair(kirin_lib):
    """eps = 0 with the r_min guard and two particles on the same spot: the guard drops that pair, the
    run stays finite, and the pair's other forces match the oracle's with the same guard."""
    p = workloads.plummer(300, 3030, eps=0.0)
    x = p.x.copy()
    x[7] = x[3]
    with abi.Kirin(p.n, 0.0, r_min=1e-6, precision="mixed") as k:
        k.set_j_particles(p.m, x, p.v)
        assert k.shared_persistent_active()
        k.hermite_init(0.0)
        st0 = k.get_state()
        k.hermite_shared_run(1.0 / 4096, 8)
        st = k.get_state()
    for key in ("x", "v", "a", "j"):
        assert np.all(np.isfinite(st[key])), key
    ref = oracle.acc_jerk_pot(p.m, x, p.v, 0.0, r_min=1e-6)
    assert np.median(metrics.rel_err_vec(st0["a"], ref[0])) <= 1e-6


def test_persistent_contexts_of_different_sizes_interleave(kirin_lib):
    """Contexts that take different group widths (N = 200, 1500, 2048) run alternately on one device;
    each run equals the same run repeated alone, bit for bit."""
    sizes = (200, 1500, 2048)
    parts = {n: workloads.plummer(n, (5050, n), eps=1.0 / 256) for n in sizes}

    def alone(n):
        p = parts[n]
        with abi.Kirin(p.n, p.eps, precision="mixed") as k:
            k.set_j_particles(p.m, p.x, p.v)
            k.hermite_init(0.0)
            k.hermite_shared_run(1.0 / 1024, 6)
            return k.get_state()

    ref = {n: alone(n) for n in sizes}
    ks = {n: abi.Kirin(parts[n].n, parts[n].eps, precision="mixed") for n in sizes}
    try:
        for n in sizes:
            ks[n].set_j_particles(parts[n].m, parts[n].x, parts[n].v)
            ks[n].hermite_init(0.0)
        for _ in range(2):
            for n in sizes:
                ks[n].hermite_shared_run(1.0 / 1024, 3)
        for n in sizes:
            st = ks[n].get_state()
            for key in ("x", "v", "a", "j", "t"):
                assert np.array_equal(st[key], ref[n][key]), (n, key)
    finally:
        for k in ks.values():
            k.close()


def test_persistent_shared_run_from_a_negative_time(kirin_lib):
    """The kernel's step times are the host's sequential sums t0 + dt + dt + ..., from any start."""
    p = workloads.plummer(512, 6060, eps=1.0 / 256)
    t0, dt, steps = -0.3, 1.0 / 1000, 7
    with abi.Kirin(p.n, p.eps, precision="mixed") as k:
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(t0)
        k.hermite_shared_run(dt, steps)
        st = k.get_state()
    t = t0
    for _ in range(steps):
        t = t + dt
    assert np.all(st["t"] == t)
    xr, vr, _, _, _ = hermite.shared_steps(p.m, p.x, p.v, p.eps, dt, steps)
    assert np.abs(st["x"] - xr).max() <= 1e-7 * np.abs(p.x).max()


def test_switching_paths_mid_run_continues_the_state(kirin_lib):
    """Five steps in the single launch, then five through the step kernels, against ten through the
    step kernels: the same state to rounding (each path leaves what the other continues from)."""
    p = workloads.plummer(1024, 7070, eps=1.0 / 256)
    dt = 1.0 / 1024
    out = []
    for first in (True, False):
        with abi.Kirin(p.n, p.eps, precision="mixed") as k:
            k.set_shared_persistent(first)
            k.set_j_particles(p.m, p.x, p.v)
            k.hermite_init(0.0)
            k.hermite_shared_run(dt, 5)
            k.set_shared_persistent(False)
            k.hermite_shared_run(dt, 5)
            out.append(k.get_state())
    assert np.all(out[0]["t"] == out[1]["t"])
    assert np.abs(out[0]["x"] - out[1]["x"]).max() <= 1e-10 * np.abs(p.x).max()
    assert np.median(metrics.rel_err_vec(out[0]["a"], out[1]["a"])) <= 1e-6


def test_persistent_shared_run_lognormal_masses_small_softening(kirin_lib):
    """Unequal (log-normal, sigma 0.5) masses and a small softening eps = 4/N: the single launch follows
    the oracle's Hermite steps, and its final forces match the oracle's at the final state."""
    n = 1500
    p = workloads.plummer(n, 8080, masses="lognormal", sigma=0.5, eps=4.0 / n)
    dt, steps = 1.0 / 2048, 8
    xr, vr, _, _, _ = hermite.shared_steps(p.m, p.x, p.v, p.eps, dt, steps)
    active, st, after = _run(p, p.eps, dt, steps, True)
    assert active
    assert np.abs(st["x"] - xr).max() <= 1e-7 * np.abs(p.x).max()
    assert np.abs(st["v"] - vr).max() <= 1e-6 * np.abs(p.v).max()
    ref = oracle.acc_jerk_pot(p.m, st["x"], st["v"], p.eps)
    for got, want in ((after[0], ref[0]), (after[1], ref[1])):
        err = metrics.rel_err_vec(got, want)
        assert np.median(err) <= 1e-6 and err.max() <= 1e-4


@pytest.mark.parametrize("persistent", [True, False])
def test_shared_run_reports_a_non_finite_state_and_recovers(kirin_lib, persistent):
    """A step so large that the predictor overflows (dt = 1e300) is reported as KIRIN_ENONFINITE by both
    paths (the single launch reports through its own error word), and the error is cleared: the same
    context then runs correctly from fresh particles."""
    p = workloads.plummer(512, 9090, eps=1.0 / 256)
    with abi.Kirin(p.n, p.eps, precision="mixed") as k:
        k.set_shared_persistent(persistent)
        k.set_j_particles(p.m, p.x, p.v)
        assert k.shared_persistent_active() == persistent
        k.hermite_init(0.0)
        with pytest.raises(abi.KirinError) as exc:
            k.hermite_shared_run(1e300, 1)
        assert exc.value.code == abi.KIRIN_ENONFINITE
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(0.0)
        k.hermite_shared_run(1.0 / 1024, 3)
        st = k.get_state()
    xr, _, _, _, _ = hermite.shared_steps(p.m, p.x, p.v, p.eps, 1.0 / 1024, 3)
    assert np.abs(st["x"] - xr).max() <= 1e-7 * np.abs(p.x).max()


@pytest.mark.parametrize("n", [2049, 3000, 4096, 6000, 8192])
def test_streamed_shared_run_matches_the_oracle(kirin_lib, n):
    """Above 2048 particles the image streams through a ring of tiles (two halves of 6 tiles): ragged and
    whole tile counts, slices of up to 54 particles per CTA (six component warps), against the oracle's
    Hermite steps and its forces at the final state."""
    p = workloads.plummer(n, (9191, n), eps=1.0 / 256)
    dt, steps = 1.0 / 1024, 6
    xr, vr, _, _, _ = hermite.shared_steps(p.m, p.x, p.v, p.eps, dt, steps)
    active, st, after = _run(p, p.eps, dt, steps, True)
    assert active
    assert np.all(st["t"] == steps * dt)
    assert np.abs(st["x"] - xr).max() <= 1e-7 * np.abs(p.x).max()
    assert np.abs(st["v"] - vr).max() <= 1e-6 * np.abs(p.v).max()
    ref = oracle.acc_jerk_pot(p.m, st["x"], st["v"], p.eps)
    err = metrics.rel_err_vec(after[0], ref[0])
    assert np.median(err) <= 1e-6 and err.max() <= 1e-4


@pytest.mark.parametrize("n,eps,r_min", [(5000, 1.0 / 256, 0.0), (4500, 0.0, 1e-6)])
def test_streamed_shared_run_agrees_with_the_kernel_path_and_itself(kirin_lib, n, eps, r_min):
    """The streamed single launch against the step kernels (to rounding), with and without the guard, and
    a run split over two calls against the same run in one call (bit for bit)."""
    p = workloads.plummer(n, 9292, eps=eps)
    dt = 1.0 / 1024
    a_on, on, _ = _run(p, eps, dt, 16, True, r_min)
    a_off, off, _ = _run(p, eps, dt, 16, False, r_min)
    assert a_on and not a_off
    assert np.all(on["t"] == off["t"])
    assert np.abs(on["x"] - off["x"]).max() <= 1e-8 * np.abs(p.x).max()
    with abi.Kirin(p.n, eps, r_min=r_min, precision="mixed") as k:
        k.set_j_particles(p.m, p.x, p.v)
        k.hermite_init(0.0)
        k.hermite_shared_run(dt, 7)
        k.hermite_shared_run(dt, 9)
        split = k.get_state()
    for key in ("x", "v", "a", "j", "t"):
        assert np.array_equal(split[key], on[key]), key
