"""Pins for the FP64 CPU oracle: values fixed by physics and mathematics, not by the oracle itself.

Each test is chosen so that a plausible slip in the oracle (a sign, a dropped
mass or G, a wrong power of s, a transposed operand, a missing factor 1/2 in
W) fails at least one of them.
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest
from scipy import integrate, spatial

import oracle
from oracle import hermite, leapfrog
from paper_0707_0438_gb300 import workloads


def icosahedron(radius):
    """The 12 vertices of a regular icosahedron (a spherical 5-design) on a sphere of given radius."""
    g = (1.0 + math.sqrt(5.0)) / 2.0
    pts = []
    for a in (-1.0, 1.0):
        for b in (-g, g):
            pts += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    pts = np.array(pts)
    return radius * pts / np.linalg.norm(pts, axis=1)[:, None]


@pytest.mark.parametrize("r_frac", [0.05, 0.1, 0.2])
def test_shell_theorem_inside(r_frac):
    """Inside a shell the pull cancels and phi = -G M / R (Newton).  A 5-design
    reproduces the shell up to Legendre order 5, so the residual is O((r/R)^5)."""
    R, M, G = 2.0, 3.0, 1.7
    shell = icosahedron(R)
    rng = np.random.default_rng(1)
    d = rng.standard_normal(3)
    probe = r_frac * R * d / np.linalg.norm(d)
    x = np.vstack([probe, shell])
    m = np.concatenate([[0.123], np.full(12, M / 12.0)])
    v = np.zeros_like(x)
    acc, jerk, pot = oracle.acc_jerk_pot(m, x, v, eps=0.0, G=G, i_idx=[0])
    scale = G * M / R ** 2
    assert np.linalg.norm(acc[0]) < 20 * r_frac ** 5 * scale
    assert abs(pot[0] - (-G * M / R)) < 5 * r_frac ** 6 * G * M / R
    assert np.all(jerk == 0.0)


@pytest.mark.parametrize("r_frac", [5.0, 10.0])
def test_shell_theorem_outside(r_frac):
    """Outside the shell it acts as a point mass at the centre: a = -G M x / r^3, phi = -G M / r."""
    R, M, G = 0.5, 2.0, 1.0
    shell = icosahedron(R)
    probe = np.array([0.3, -0.4, 1.2])
    probe = r_frac * R * probe / np.linalg.norm(probe)
    x = np.vstack([shell, probe])
    m = np.concatenate([np.full(12, M / 12.0), [1.0]])
    acc, _, pot = oracle.acc_jerk_pot(m, x, np.zeros_like(x), 0.0, G, i_idx=[12])
    r = np.linalg.norm(probe)
    expect = -G * M * probe / r ** 3
    assert np.linalg.norm(acc[0] - expect) < 20 * (1 / r_frac) ** 6 * np.linalg.norm(expect)
    assert abs(pot[0] + G * M / r) < 5 * (1 / r_frac) ** 7 * G * M / r


def test_attraction_sign_and_softening_two_body():
    """Two bodies on the x axis: the lighter one is pulled towards the heavier with G m2 d / (d^2+eps^2)^(3/2)."""
    G, eps = 2.0, 0.3
    m = np.array([1.0, 4.0])
    x = np.array([[0.0, 0.0, 0.0], [1.5, 0.0, 0.0]])
    v = np.array([[0.0, 0.0, 0.0], [0.0, 0.2, 0.0]])
    acc, jerk, pot = oracle.acc_jerk_pot(m, x, v, eps, G)
    s = math.sqrt(1.5 ** 2 + eps ** 2)
    assert acc[0, 0] == pytest.approx(G * 4.0 * 1.5 / s ** 3, rel=1e-15)
    assert acc[1, 0] == pytest.approx(-G * 1.0 * 1.5 / s ** 3, rel=1e-15)
    assert pot[0] == pytest.approx(-G * 4.0 / s, rel=1e-15)
    assert pot[1] == pytest.approx(-G * 1.0 / s, rel=1e-15)
    # relative motion purely transverse: d.w = 0, so jerk_0 = G m_1 w / s^3
    assert jerk[0, 1] == pytest.approx(G * 4.0 * 0.2 / s ** 3, rel=1e-15)
    assert jerk[0, 0] == 0.0 and jerk[0, 2] == 0.0


def test_newton_third_law():
    p = workloads.plummer(512, 77, masses="lognormal")
    acc, jerk, _ = oracle.acc_jerk_pot(p.m, p.x, p.v, 0.01)
    ma = p.m[:, None] * acc
    mj = p.m[:, None] * jerk
    assert np.linalg.norm(ma.sum(0)) < 1e-14 * np.abs(ma).sum()
    assert np.linalg.norm(mj.sum(0)) < 1e-14 * np.abs(mj).sum()


@pytest.mark.parametrize("eps", [0.0, 0.02])
def test_jerk_is_time_derivative_of_acc(eps):
    """jerk = d/dt a(x + v t) at t = 0; central differences converge as h^2."""
    p = workloads.plummer(64, 5)
    acc_at = lambda h: oracle.acc_jerk_pot(p.m, p.x + h * p.v, p.v, eps)[0]
    _, jerk, _ = oracle.acc_jerk_pot(p.m, p.x, p.v, eps)
    errs = []
    for h in (2e-5, 1e-5):
        fd = (acc_at(h) - acc_at(-h)) / (2 * h)
        errs.append(np.linalg.norm(fd - jerk) / np.linalg.norm(jerk))
    assert errs[1] < 5e-6
    assert 3.0 < errs[0] / errs[1] < 5.0  # second-order convergence


def test_acc_is_minus_gradient_of_potential_energy():
    """dW/dx_k = -m_k a_k for W = 1/2 sum m_i phi_i: ties the potential to the force."""
    p = workloads.plummer(32, 9, masses="lognormal")
    eps, G, h = 0.05, 1.3, 1e-6
    acc, _, _ = oracle.acc_jerk_pot(p.m, p.x, p.v, eps, G)
    for k in (0, 7, 31):
        for c in range(3):
            xp, xm = p.x.copy(), p.x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            dW = (oracle.energy(p.m, xp, p.v, eps, G)[1] - oracle.energy(p.m, xm, p.v, eps, G)[1]) / (2 * h)
            assert dW == pytest.approx(-p.m[k] * acc[k, c], rel=1e-6, abs=1e-9)


def test_energy_kinetic_and_pot_consistency():
    p = workloads.plummer(128, 3)
    kin, w = oracle.energy(p.m, p.x, p.v, 0.01)
    _, _, pot = oracle.acc_jerk_pot(p.m, p.x, p.v, 0.01)
    assert kin == pytest.approx(0.5 * np.sum(p.m * np.sum(p.v * p.v, axis=1)), rel=1e-14)
    assert w == pytest.approx(0.5 * np.sum(p.m * pot), rel=1e-13)


def _plummer_pair_mean_inverse_distance(trunc):
    """E[1/|r1 - r2|] for two independent points of a Plummer sphere (a = 1) truncated at mass
    fraction trunc.  By the shell theorem E[1/|r1-r2| given radii] = 1/max(r1, r2), so
    E = (2/f^2) int_0^rmax p(r) F(r) / r dr = (6/f^2) int_0^rmax r^4 / (1 + r^2)^4 dr;
    untruncated this is 3 pi / 16 and W = -3 pi / 32 (G = M = a = 1)."""
    rmax = (trunc ** (-2.0 / 3.0) - 1.0) ** -0.5
    val, _ = integrate.quad(lambda r: r ** 4 / (1 + r * r) ** 4, 0.0, rmax, epsabs=1e-14, epsrel=1e-13)
    return 6.0 * val / trunc ** 2


def test_plummer_closed_form_integral():
    full, _ = integrate.quad(lambda r: r ** 4 / (1 + r * r) ** 4, 0.0, np.inf)
    assert 6.0 * full == pytest.approx(3 * math.pi / 16, rel=1e-12)


@pytest.mark.parametrize("henon", [False, True])
def test_plummer_potential_energy(henon):
    """Potential energy of an equal-mass Plummer sample at eps = 0 against the closed form
    -(1 - 1/N) E[1/r12] / 2  (-3 pi / 32 (1 - 1/N) untruncated, a = 1 units; -1/2 (1 - 1/N) in Henon units)."""
    n, seeds = 2048, range(8)
    ws = []
    for s in seeds:
        p = workloads.plummer(n, (4242, s), henon=henon)
        ws.append(oracle.energy(p.m, p.x, p.v, 0.0)[1])
    ws = np.array(ws)
    e_inv = _plummer_pair_mean_inverse_distance(0.999)
    if henon:
        e_inv /= workloads.HENON_R
    expect = -0.5 * (1.0 - 1.0 / n) * e_inv
    sigma = ws.std(ddof=1) / math.sqrt(len(ws))
    assert abs(ws.mean() - expect) < 4 * sigma + 1e-3 * abs(expect)
    # and the truncation moves the expectation by only ~0.2 %
    untrunc = -3 * math.pi / 32 * (1 - 1 / n) / (workloads.HENON_R if henon else 1.0)
    assert abs(expect / untrunc - 1) < 3e-3


def test_plummer_virial():
    """Virial equilibrium 2K + W = 0 of the Henon-scaled sample (within sampling noise)."""
    ratios = []
    for s in range(6):
        p = workloads.plummer(2048, (99, s))
        k, w = oracle.energy(p.m, p.x, p.v, 0.0)
        ratios.append(2 * k / -w)
    assert abs(np.mean(ratios) - 1.0) < 0.03


def _decimal_brute_force(m, x, v, eps, G, prec=40):
    getcontext().prec = prec
    D = lambda a: Decimal(repr(float(a)))
    n = len(m)
    out = []
    for i in range(n):
        a = [Decimal(0)] * 3
        jk = [Decimal(0)] * 3
        p = Decimal(0)
        for j in range(n):
            if j == i:
                continue
            d = [D(x[j][c]) - D(x[i][c]) for c in range(3)]
            w = [D(v[j][c]) - D(v[i][c]) for c in range(3)]
            s2 = sum(dc * dc for dc in d) + D(eps) * D(eps)
            s = s2.sqrt()
            s3 = s2 * s
            dw = sum(d[c] * w[c] for c in range(3))
            for c in range(3):
                a[c] += D(m[j]) * d[c] / s3
                jk[c] += D(m[j]) * (w[c] / s3 - 3 * dw * d[c] / (s3 * s2))
            p -= D(m[j]) / s
        out.append(([float(D(G) * q) for q in a], [float(D(G) * q) for q in jk], float(D(G) * p)))
    return out


def test_fp64_rounding_against_40_digit_sum():
    """At N = 12 the FP64 oracle agrees with a 40-digit decimal evaluation to a few ulp."""
    p = workloads.plummer(12, 31, masses="lognormal")
    acc, jerk, pot = oracle.acc_jerk_pot(p.m, p.x, p.v, 0.01, 1.0)
    ref = _decimal_brute_force(p.m, p.x, p.v, 0.01, 1.0)
    for k, (a, j, ph) in enumerate(ref):
        assert np.linalg.norm(acc[k] - a) <= 1e-14 * np.linalg.norm(a)
        assert np.linalg.norm(jerk[k] - j) <= 1e-13 * np.linalg.norm(j)
        assert abs(pot[k] - ph) <= 1e-15 * abs(ph)


def test_translation_rotation_permutation_invariance():
    p = workloads.plummer(200, 12, masses="lognormal")
    eps = 0.01
    acc, jerk, pot = oracle.acc_jerk_pot(p.m, p.x, p.v, eps)
    # translation of all positions / Galilean boost of all velocities
    acc2, jerk2, pot2 = oracle.acc_jerk_pot(p.m, p.x + np.array([0.25, -0.5, 1.0]), p.v + 0.3, eps)
    assert np.allclose(acc2, acc, rtol=0, atol=1e-12 * np.abs(acc).max())
    assert np.allclose(jerk2, jerk, rtol=0, atol=1e-12 * np.abs(jerk).max())
    assert np.allclose(pot2, pot, rtol=1e-13)
    # rotation
    q, _ = np.linalg.qr(np.random.default_rng(4).standard_normal((3, 3)))
    acc3, jerk3, pot3 = oracle.acc_jerk_pot(p.m, p.x @ q.T, p.v @ q.T, eps)
    assert np.allclose(acc3, acc @ q.T, atol=1e-12 * np.abs(acc).max())
    assert np.allclose(jerk3, jerk @ q.T, atol=1e-12 * np.abs(jerk).max())
    assert np.allclose(pot3, pot, rtol=1e-13)
    # relabelling the particles permutes the results
    perm = np.random.default_rng(5).permutation(p.n)
    acc4, jerk4, pot4 = oracle.acc_jerk_pot(p.m[perm], p.x[perm], p.v[perm], eps)
    assert np.allclose(acc4, acc[perm], atol=1e-13 * np.abs(acc).max())
    assert np.allclose(pot4, pot[perm], rtol=1e-14)


def test_homogeneity_under_scaling():
    """Dimensional homogeneity of Eq. 1 and its time derivative: x -> lam x, eps -> lam eps, m -> mu m,
    v -> nu v, G -> g G give a -> g mu a / lam^2, phi -> g mu phi / lam, jerk -> g mu nu jerk / lam^3.
    With powers of two every floating-point step scales exactly, so the oracle must reproduce the
    scaling bit for bit; a wrong power of s, of the separation or of the mass anywhere breaks it."""
    p = workloads.plummer(60, 808, masses="lognormal", eps=0.02)
    a, j, f = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps)
    for lam, mu, nu, g in ((2.0 ** -3, 2.0 ** 5, 2.0 ** 2, 1.0), (2.0 ** 4, 2.0 ** -7, 2.0 ** -3, 0.5)):
        a2, j2, f2 = oracle.acc_jerk_pot(mu * p.m, lam * p.x, nu * p.v, lam * p.eps, G=g)
        assert np.array_equal(a2, g * mu / lam ** 2 * a)
        assert np.array_equal(f2, g * mu / lam * f)
        assert np.array_equal(j2, g * mu * nu / lam ** 3 * j)
    # a factor that is not a power of two: equal to rounding
    lam, mu, nu = 1.7, 0.3, 2.9
    a2, j2, f2 = oracle.acc_jerk_pot(mu * p.m, lam * p.x, nu * p.v, lam * p.eps)
    assert np.allclose(a2, mu / lam ** 2 * a, rtol=1e-13, atol=0)
    assert np.allclose(f2, mu / lam * f, rtol=1e-13, atol=0)
    assert np.allclose(j2, mu * nu / lam ** 3 * j, rtol=1e-12, atol=1e-12 * np.abs(j).max())


def test_i_subset_equals_full_rows():
    p = workloads.plummer(300, 8)
    acc, jerk, pot = oracle.acc_jerk_pot(p.m, p.x, p.v, 0.01)
    idx = np.array([299, 0, 17, 17, 150])
    a2, j2, p2 = oracle.acc_jerk_pot(p.m, p.x, p.v, 0.01, i_idx=idx)
    assert np.array_equal(a2, acc[idx]) and np.array_equal(j2, jerk[idx]) and np.array_equal(p2, pot[idx])


def test_zero_softening_guard():
    """eps = 0: a coincident distinct pair contributes nothing; s^2 is raised to r_min^2 (Sect. 3.3.1)."""
    m = np.array([1.0, 2.0, 3.0, 0.5])
    x = np.array([[0, 0, 0], [0, 0, 0], [1e-8, 0, 0], [2.0, 0, 0]], dtype=float)
    v = np.zeros_like(x)
    acc, _, pot = oracle.acc_jerk_pot(m, x, v, 0.0, r_min=1e-6, i_idx=[0])
    expect_x = 3.0 * 1e-8 / 1e-18 + 0.5 * 2.0 / 8.0
    assert acc[0, 0] == pytest.approx(expect_x, rel=1e-14)
    assert pot[0] == pytest.approx(-3.0 / 1e-6 - 0.5 / 2.0, rel=1e-14)


def test_adjoint_matches_finite_differences():
    """dL/dx, dL/dm of L = sum_i g_i . a_i(x, m) against central differences."""
    p = workloads.plummer(16, 21, masses="lognormal")
    eps, G, h = 0.1, 1.0, 1e-6
    g = np.random.default_rng(2).standard_normal((16, 3))
    L = lambda m, x: float(np.sum(g * oracle.acc_pot(m, x, eps, G)[0]))
    gx, gm = oracle.force_adjoint(p.m, p.x, g, eps, G)
    for k in range(16):
        for c in range(3):
            xp, xm = p.x.copy(), p.x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            assert gx[k, c] == pytest.approx((L(p.m, xp) - L(p.m, xm)) / (2 * h), rel=1e-6, abs=1e-7)
        mp, mm = p.m.copy(), p.m.copy()
        mp[k] += h
        mm[k] -= h
        assert gm[k] == pytest.approx((L(mp, p.x) - L(mm, p.x)) / (2 * h), rel=1e-6, abs=1e-7)


def test_leapfrog_adjoint_matches_finite_differences():
    p = workloads.plummer(16, 23)
    eps, dt, steps = 0.05, 1.0 / 64, 8
    tgt = p.x + 0.01
    L, gx, gv, gm = leapfrog.loss_grad(p.m, p.x, p.v, eps, dt, steps, tgt)
    h = 1e-6
    rng = np.random.default_rng(3)
    for _ in range(6):
        k, c = rng.integers(16), rng.integers(3)
        for arr, grad in ((p.x, gx), (p.v, gv)):
            ap, am = arr.copy(), arr.copy()
            ap[k, c] += h
            am[k, c] -= h
            if arr is p.x:
                fd = (leapfrog.loss(p.m, ap, p.v, eps, dt, steps, tgt) - leapfrog.loss(p.m, am, p.v, eps, dt, steps, tgt)) / (2 * h)
            else:
                fd = (leapfrog.loss(p.m, p.x, ap, eps, dt, steps, tgt) - leapfrog.loss(p.m, p.x, am, eps, dt, steps, tgt)) / (2 * h)
            assert grad[k, c] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        mp, mm = p.m.copy(), p.m.copy()
        mp[k] += h
        mm[k] -= h
        fd = (leapfrog.loss(mp, p.x, p.v, eps, dt, steps, tgt) - leapfrog.loss(mm, p.x, p.v, eps, dt, steps, tgt)) / (2 * h)
        assert gm[k] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def _kepler_relative(t, a, e, period):
    """Relative position of a Kepler orbit started at pericentre (solve M = E - e sin E by Newton)."""
    M = 2 * math.pi * t / period
    E = M
    for _ in range(60):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


def _two_body(e=0.5, a=1.0):
    m = np.array([0.5, 0.5])
    rp = a * (1 - e)
    vp = math.sqrt((1 + e) / (a * (1 - e)))
    rel_x = np.array([rp, 0, 0])
    rel_v = np.array([0, vp, 0])
    x = np.vstack([-0.5 * rel_x, 0.5 * rel_x])
    v = np.vstack([-0.5 * rel_v, 0.5 * rel_v])
    return m, x, v


def test_hermite_kepler_orbit_fourth_order():
    """Hermite shared steps on a two-body e = 0.5 orbit match Kepler's equation, error ~ dt^4."""
    m, x, v = _two_body()
    period = 2 * math.pi
    t_end = period / 2
    errs = []
    for n_steps in (256, 512):
        dt = t_end / n_steps
        xf, vf, _, _, _ = hermite.shared_steps(m, x, v, 0.0, dt, n_steps)
        rel = xf[1] - xf[0]
        errs.append(np.linalg.norm(rel - _kepler_relative(t_end, 1.0, 0.5, period)))
    assert errs[0] < 1e-6
    ratio = errs[0] / errs[1]
    assert 10.0 < ratio < 24.0


def test_hermite_block_steps_conserve_energy_and_sync():
    p = workloads.plummer(96, 17)
    out = hermite.block_steps(p.m, p.x, p.v, 0.01, t_end=1.0 / 8.0)
    assert np.all(out["t"] == 1.0 / 8.0)
    lv = np.log2(out["dt"])
    assert np.all(lv == np.round(lv)) and lv.min() >= -20 and lv.max() <= -3
    assert abs(out["dE_E"]) < 1e-5
    assert sum(out["blocks"]) >= p.n


def test_block_steps_with_one_level_are_shared_steps(monkeypatch):
    """With dt_min = dt_max the block scheduler must select every particle at every step: the block
    integrator then reduces exactly to the shared-step one (itself pinned on the Kepler orbit)."""
    p = workloads.plummer(64, 19, eps=0.01)
    dt = 2.0 ** -8
    monkeypatch.setattr(hermite, "DT_MIN", dt)
    monkeypatch.setattr(hermite, "DT_MAX", dt)
    out = hermite.block_steps(p.m, p.x, p.v, p.eps, t_end=16 * dt)
    x, v, a, j, _ = hermite.shared_steps(p.m, p.x, p.v, p.eps, dt, 16)
    assert out["blocks"] == [p.n] * 16
    assert np.all(out["t"] == 16 * dt) and np.all(out["dt"] == dt)
    for got, ref in ((out["x"], x), (out["v"], v)):
        assert np.array_equal(got, ref)


def test_leapfrog_is_time_reversible():
    """Kick-drift-kick is symmetric in time: n steps forward, velocities negated, n steps forward again
    return the initial state up to rounding.  A wrong kick/drift order or half-kick weight breaks it."""
    p = workloads.plummer(64, 23, eps=0.05)
    xs, vs = leapfrog.trajectory(p.m, p.x, p.v, p.eps, 1.0 / 64, 32)
    xb, vb = leapfrog.trajectory(p.m, xs[-1], -vs[-1], p.eps, 1.0 / 64, 32)
    assert np.abs(xb[-1] - p.x).max() <= 1e-12 * np.abs(p.x).max()
    assert np.abs(-vb[-1] - p.v).max() <= 1e-12 * np.abs(p.v).max()
    # and the motion in between is real
    assert np.abs(xs[-1] - p.x).max() > 1e-3


def test_nearest_neighbour_matches_kdtree():
    p = workloads.plummer(500, 41)
    idx = np.arange(0, 500, 7)
    nn, r2 = oracle.nearest(p.x, idx)
    d, k = spatial.cKDTree(p.x).query(p.x[idx], k=2)
    assert np.array_equal(nn, k[:, 1])
    assert np.allclose(np.sqrt(r2), d[:, 1], rtol=1e-14)


# ---- acceleration + potential without jerk (the leapfrog clients of Sect. 4.3) ----

@pytest.mark.parametrize("eps", [0.0, 0.01])
def test_acc_pot_equals_acc_jerk_pot_bit_for_bit(eps):
    """oracle.acc_pot forms the same separations, s^3 and 1/s terms in the same j order as
    acc_jerk_pot (itself pinned above), so its acceleration and potential must be identical
    bits.  A sign slip, a dropped G or mass, or a wrong power of s in either potential or
    acceleration of acc_pot breaks the equality."""
    p = workloads.plummer(300, 61, masses="lognormal")
    idx = np.array([0, 299, 17, 150, 17, 3])
    for G in (1.0, 0.7):
        a_ref, _, p_ref = oracle.acc_jerk_pot(p.m, p.x, p.v, eps, G, i_idx=idx)
        a, ph = oracle.acc_pot(p.m, p.x, eps, G, i_idx=idx)
        assert np.array_equal(a, a_ref) and np.array_equal(ph, p_ref)
    a_all, p_all = oracle.acc_pot(p.m, p.x, eps)
    a_ref, _, p_ref = oracle.acc_jerk_pot(p.m, p.x, p.v, eps)
    assert np.array_equal(a_all, a_ref) and np.array_equal(p_all, p_ref)


def test_acc_pot_skips_a_coincident_pair_at_zero_softening():
    """eps = 0 and a distinct particle at the same place: that pair contributes nothing (Sect. 3.3.1),
    the others their point-mass terms, written out by hand."""
    m = np.array([1.0, 2.0, 0.5])
    x = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, -4.0, 0.0]])
    a, ph = oracle.acc_pot(m, x, 0.0, G=3.0, i_idx=[0])
    assert np.array_equal(a[0], np.array([0.0, -3.0 * 0.5 * 4.0 / 64.0, 0.0]))
    assert ph[0] == -3.0 * 0.5 / 4.0


@pytest.mark.parametrize("r_frac", [0.05, 0.2])
def test_acc_pot_shell_theorem(r_frac):
    """The shell theorem through acc_pot: inside, a = 0 and phi = -G M / R up to O((r/R)^5); outside,
    a point mass at the centre.  Pins the potential's sign, G and mass factor independently of the
    jerk-carrying routine."""
    R, M, G = 2.0, 3.0, 1.7
    shell = icosahedron(R)
    d = np.array([0.6, -0.3, 0.74])
    probe = r_frac * R * d / np.linalg.norm(d)
    m = np.concatenate([[0.123], np.full(12, M / 12.0)])
    acc, pot = oracle.acc_pot(m, np.vstack([probe, shell]), 0.0, G, i_idx=[0])
    assert np.linalg.norm(acc[0]) < 20 * r_frac ** 5 * G * M / R ** 2
    assert abs(pot[0] + G * M / R) < 5 * r_frac ** 6 * G * M / R
    far = probe / r_frac * 5.0 / 1.0  # at 5 R
    acc, pot = oracle.acc_pot(m, np.vstack([far, shell]), 0.0, G, i_idx=[0])
    r = np.linalg.norm(far)
    expect = -G * M * far / r ** 3
    assert np.linalg.norm(acc[0] - expect) < 20 * 0.2 ** 6 * np.linalg.norm(expect)
    assert abs(pot[0] + G * M / r) < 5 * 0.2 ** 7 * G * M / r


# ---- Aarseth's time-step criterion (Sect. 3: the Makino & Aarseth Hermite scheme) ----

def _circular_binary(G=1.3, m1=0.25, m2=0.75, d=2.0):
    """Two bodies on a circular orbit of separation d about their centre of mass: angular rate
    omega = sqrt(G (m1 + m2) / d^3), radii d m2 / M and d m1 / M."""
    M = m1 + m2
    w = math.sqrt(G * M / d ** 3)
    r1, r2 = d * m2 / M, d * m1 / M
    m = np.array([m1, m2])
    x = np.array([[r1, 0.0, 0.0], [-r2, 0.0, 0.0]])
    v = np.array([[0.0, w * r1, 0.0], [0.0, -w * r2, 0.0]])
    return m, x, v, G, w


def test_aarseth_step_on_exact_circular_derivatives():
    """On a circular orbit of rate omega, |a| = omega^2 r, |jerk| = omega^3 r, |a2| = omega^4 r and
    |a3| = omega^5 r, so both products in the numerator and in the denominator are equal and the
    criterion gives exactly sqrt(eta) / omega.  Catches a missing square root, eta inside the root
    twice or not at all, and a wrong power of any derivative."""
    for w, r, eta in ((1.0, 0.5, 0.01), (0.37, 3.0, 0.02), (5.0, 1e-3, 0.003)):
        ph = 0.8
        x = r * np.array([math.cos(ph), math.sin(ph), 0.0])
        u = r * w * np.array([-math.sin(ph), math.cos(ph), 0.0])   # velocity
        a1, j1 = -w * w * x, -w * w * u
        a2, a3 = w ** 4 * x, w ** 4 * u
        got = hermite.aarseth_step(a1[None], j1[None], a2[None], a3[None], np.array([0.0]), eta)
        assert got[0] == pytest.approx(math.sqrt(eta) / w, rel=1e-14)


def test_aarseth_step_after_one_hermite_step_on_a_circular_orbit():
    """One shared Hermite step of the oracle on a circular binary, then the derivatives the corrector
    interpolates: the criterion returns sqrt(eta) / omega up to O((omega dt)^2), and the error falls
    by about 4 when dt halves."""
    m, x, v, G, w = _circular_binary()
    eta = 0.01
    errs = []
    for wdt in (0.02, 0.01):
        dt = wdt / w
        _, _, _, _, ev = hermite.shared_steps(m, x, v, 0.0, dt, 1, G=G)
        (a0, j0, _), (a1, j1, _) = ev
        a2, a3 = hermite.hermite_derivatives(a0, j0, a1, j1, dt)
        got = hermite.aarseth_step(a1, j1, a2, a3, dt, eta)
        e = np.abs(got * w / math.sqrt(eta) - 1.0)
        assert np.all(e < wdt ** 2)
        errs.append(e.max())
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_aarseth_step_hand_computed_non_parallel_vectors():
    """Hand-worked rows with derivatives in different directions, where the terms of the criterion
    differ.  Row 1: |a1| = 5, |jerk| = 2, a2 carried to the end of the step a2 + dt a3 = (2, 0, 1)
    with |.| = sqrt(5), |a3| = 2 sqrt(2):  dt = sqrt(eta (5 sqrt 5 + 4) / (4 sqrt 2 + 5)).
    Row 2 (its own dt = 0.25): a2 + dt a3 = (0, 3, 0) + (0, 1, 0) = (0, 4, 0), |a1| = 13 from
    (5, 12, 0), |jerk| = 1, |a3| = 4:  dt = sqrt(eta (13 * 4 + 1) / (1 * 4 + 16)).
    Not carrying a2 to the end of the step, carrying it with the wrong sign, or exchanging any two
    of the four terms changes both rows."""
    eta = 0.01
    a1 = np.array([[3.0, 0.0, 4.0], [5.0, 12.0, 0.0]])
    j1 = np.array([[0.0, 2.0, 0.0], [0.0, 0.0, -1.0]])
    a2 = np.array([[1.0, 0.0, 0.0], [0.0, 3.0, 0.0]])
    a3 = np.array([[2.0, 0.0, 2.0], [0.0, 4.0, 0.0]])
    dt = np.array([0.5, 0.25])
    got = hermite.aarseth_step(a1, j1, a2, a3, dt, eta)
    assert got[0] == pytest.approx(math.sqrt(eta * (5 * math.sqrt(5) + 4) / (4 * math.sqrt(2) + 5)), rel=1e-15)
    assert got[1] == pytest.approx(math.sqrt(eta * 53.0 / 20.0), rel=1e-15)
