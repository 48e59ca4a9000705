"""GPU parity of the direct sum (acc, jerk, pot) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_0707_0438_gb300 import abi, metrics, workloads
from tests.gpu_util import TOL, assert_parity, errors

pytestmark = pytest.mark.gpu

PRECISIONS = ["mixed", "fp64"]


def _ctx(p, precision, r_min=0.0, n_max=None):
    k = abi.Kirin(n_max or max(p.n, 1), p.eps, r_min=r_min, precision=precision)
    k.set_j_particles(p.m, p.x, p.v)
    return k


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n", [2, 3, 100, 1000, 1024, 2049, 5000])
def test_full_evaluation_matches_oracle(kirin_lib, precision, n):
    """All i against all j, sizes spanning one tile, several tiles and ragged tails."""
    p = workloads.plummer(n, (1001, n), eps=1.0 / 256.0)
    with _ctx(p, precision) as k:
        got = k.forces()
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps)
    assert_parity(got, ref, precision, f"N={n}")


@pytest.mark.parametrize("precision", PRECISIONS)
def test_single_particle_has_no_force(kirin_lib, precision):
    p = workloads.plummer(1, 5, eps=0.01)
    with _ctx(p, precision) as k:
        acc, jerk, pot = k.forces()
    assert np.all(acc == 0) and np.all(jerk == 0) and np.all(pot == 0)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n_i", [1, 31, 32, 127, 511, 4095, 4096, 8192])
def test_active_blocks_of_every_size(kirin_lib, precision, n_i):
    """Block-step active lists from 1 particle to all: exercises the j-groups and the j-split (Sect. 3.2)."""
    p = workloads.plummer(8192, 1002, eps=1e-3)
    il = workloads.i_subset(p.n, n_i, seed=n_i)
    with _ctx(p, precision) as k:
        got = k.forces(il)
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    assert_parity(got, ref, precision, f"n_i={n_i}")


@pytest.mark.parametrize("precision", PRECISIONS)
def test_every_launch_shape_gives_the_same_answer(kirin_lib, precision):
    p = workloads.plummer(3000, 77, masses="lognormal", eps=0.005)
    il = workloads.i_subset(p.n, 700, seed=3)
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    results = []
    with _ctx(p, precision) as k:
        for groups in (1, 2, 4, 8):
            for n_split in (1, 2, 3, 7, 24):
                k.set_launch(groups, n_split)
                got = k.forces(il)
                assert_parity(got, ref, precision, f"groups={groups} split={n_split}")
                results.append(got)
        k.set_launch(0, 0)
    if precision == "fp64":
        # different splits only reorder an FP64 sum: vectors agree to a few ulp of their norm
        for got in results[1:]:
            assert np.max(metrics.rel_err_vec(got[0], results[0][0])) <= 1e-13


@pytest.mark.parametrize("precision", PRECISIONS)
def test_wide_j_split_reduction(kirin_lib, precision):
    """Few i against many j tiles with up to one split per tile (Sect. 3.2): the
    split partials are reduced by 1 to 32 lanes per output."""
    p = workloads.plummer(40000, 91, eps=1e-3)  # 313 tiles, the last one ragged
    il = workloads.i_subset(p.n, 37, seed=5)
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    with _ctx(p, precision) as k:
        for groups, n_split in ((8, 9), (8, 64), (4, 130), (1, 257), (8, 1024)):
            k.set_launch(groups, n_split)
            assert_parity(k.forces(il), ref, precision, f"groups={groups} split={n_split}")
        k.set_launch(0, 0)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_empty_i_list(kirin_lib, precision):
    """No active i: the host call returns empty results, the device call does nothing."""
    import torch
    p = workloads.plummer(500, 31, eps=0.01)
    with _ctx(p, precision) as k:
        acc, jerk, pot = k.forces(np.zeros(0, dtype=np.int32))
        assert acc.shape == (0, 3) and jerk.shape == (0, 3) and pot.shape == (0,)
        dev = torch.device("cuda:0")
        out = torch.full((4, 3), 7.0, dtype=torch.float64, device=dev)
        k.compute_forces_dev(torch.zeros(0, dtype=torch.int32, device=dev), out, out, out[:, 0])
        k.sync()
        assert bool((out == 7.0).all())
        acc, _, _ = k.forces(np.array([3], dtype=np.int32))  # the context is still usable
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=np.array([3]))
    assert np.allclose(acc, ref[0], rtol=1e-5)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_far_from_the_origin(kirin_lib, precision):
    """A cluster at |x| ~ 1e4 with separations down to ~1e-3: the FP32 high parts of the positions are
    2^-10 apart there, so only the double-single separation (high parts subtracted exactly, low parts
    added) keeps the mixed forces within the stated tolerance."""
    p = workloads.plummer(2000, 33, eps=1e-3)
    x = p.x + np.array([1.0e4, -0.7e4, 0.3e4])
    ref = oracle.acc_jerk_pot(p.m, x, p.v, p.eps)
    with abi.Kirin(p.n, p.eps, precision=precision) as k:
        k.set_j_particles(p.m, x, p.v)
        got = k.forces()
    assert_parity(got, ref, precision, "offset 1e4")
    # and the forces are those of the cluster at the origin (translation invariance)
    at0 = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps)
    assert np.median(metrics.rel_err_vec(got[0], at0[0])) <= (1e-6 if precision == "mixed" else 1e-10)


def test_maximum_size_sampled_parity(kirin_lib):
    """N = 2^25 (about 15 GB on the device; image offsets and tile indices far beyond 2^24): 256
    sampled i, the last particle among them, against the oracle over all j."""
    p = workloads.gaussian_cloud(1 << 25, 2025, eps=1e-4)
    il = workloads.i_subset(p.n, 256, seed=25)
    il[-1] = p.n - 1
    with _ctx(p, "mixed") as k:
        got = k.forces(il)
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    assert_parity(got, ref, "mixed", "N=2^25")


@pytest.mark.parametrize("n_i", [1, 2, 5, 8])
def test_tiny_block_kernel(kirin_lib, n_i):
    """Blocks of at most 8 i go to the tiny-block kernel (j ranges per CTA, lanes over j, Sect. 3.2's
    j-split taken to the limit); ragged j count, the self pair inside the list, and agreement with the
    regular kernel under a fixed launch shape."""
    p = workloads.plummer(40000, 93, masses="lognormal", eps=1e-3)  # 313 tiles, the last one ragged
    il = workloads.i_subset(p.n, n_i, seed=n_i)
    il[0] = p.n - 1  # the last particle, in the ragged tile
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    with _ctx(p, "mixed") as k:
        assert k.get_launch(n_i)[0] == 0 and k.get_launch(9)[0] != 0
        tiny = k.forces(il)
        k.set_launch(8, 64)
        regular = k.forces(il)
        k.set_launch(0, 0)
    assert_parity(tiny, ref, "mixed", f"tiny n_i={n_i}")
    for a, b in zip(tiny, regular):
        assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))


def test_tiny_block_kernel_guard_and_duplicates(kirin_lib):
    """eps = 0 with r_min through the tiny-block kernel: a coincident distinct pair contributes
    nothing, repeated and unordered i are each evaluated."""
    p = workloads.plummer(3001, 94, eps=0.0)
    x = p.x.copy()
    x[7] = x[8]
    r_min = 1e-6
    il = np.array([8, 3000, 7, 8, 0, 1500], dtype=np.int32)
    with abi.Kirin(p.n, 0.0, r_min=r_min, precision="mixed") as k:
        k.set_j_particles(p.m, x, p.v)
        assert k.get_launch(len(il))[0] == 0
        got = k.forces(il)
    ref = oracle.acc_jerk_pot(p.m, x, p.v, 0.0, r_min=r_min, i_idx=il)
    assert_parity(got, ref, "mixed", "tiny eps=0")
    assert np.array_equal(got[0][0], got[0][3])


@pytest.mark.parametrize("precision", PRECISIONS)
def test_duplicate_and_unordered_i_list(kirin_lib, precision):
    p = workloads.plummer(700, 8, eps=0.01)
    il = np.array([699, 0, 17, 17, 350, 0], dtype=np.int32)
    with _ctx(p, precision) as k:
        got = k.forces(il)
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    assert_parity(got, ref, precision)
    assert np.array_equal(got[0][2], got[0][3])


@pytest.mark.parametrize("precision", PRECISIONS)
def test_lognormal_masses_and_tiny_softening(kirin_lib, precision):
    """The large-N workload's mass spectrum and eps = 4/N, at a size the oracle does in a second."""
    n = 16384
    p = workloads.plummer(n, 1003, masses="lognormal", eps=4.0 / n)
    il = workloads.i_subset(n, 2048, seed=5)
    with _ctx(p, precision) as k:
        got = k.forces(il)
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    assert_parity(got, ref, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_zero_softening_guard(kirin_lib, precision):
    """eps = 0 with r_min: coincident distinct particles contribute nothing (Sect. 3.3.1)."""
    p = workloads.plummer(1500, 31, eps=0.0)
    x = p.x.copy()
    x[10] = x[11]                    # a coincident pair
    x[20] = x[21] + 1e-9             # a pair closer than r_min
    x[30] = x[31] + 3e-3             # a close pair above r_min
    r_min = 1e-6
    with abi.Kirin(p.n, 0.0, r_min=r_min, precision=precision) as k:
        k.set_j_particles(p.m, x, p.v)
        got = k.forces()
    ref = oracle.acc_jerk_pot(p.m, x, p.v, 0.0, r_min=r_min)
    errs = errors(got, ref)
    med, mx = TOL[precision]["acc"]
    assert errs["acc"]["median"] <= med, errs
    # the pair at 1e-9 sits below the floor in double-single; its force is
    # m / r_min^2-sized and dominates: compare those two particles separately
    keep = np.ones(p.n, bool)
    keep[[20, 21]] = False
    sub = tuple(q[keep] for q in got), tuple(q[keep] for q in ref)
    assert_parity(*sub, precision, "eps=0")
    for i in (20, 21):
        assert np.linalg.norm(got[0][i] - ref[0][i]) <= 1e-3 * np.linalg.norm(ref[0][i])
    assert np.all(np.isfinite(got[0])) and np.all(np.isfinite(got[2]))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_predictor_on_device(kirin_lib, precision):
    """GPU_set_ti: predicted positions/velocities (FP64 Taylor series) feed the force."""
    p = workloads.plummer(2000, 42, eps=0.01)
    rng = np.random.default_rng(0)
    a = rng.standard_normal((p.n, 3))
    j = rng.standard_normal((p.n, 3))
    t0 = rng.uniform(0.0, 0.01, p.n)
    t = 0.0123
    with abi.Kirin(p.n, p.eps, precision=precision) as k:
        k.set_j_particles(p.m, p.x, p.v, a, j, t0)
        k.predict(t)
        got = k.forces()
    dt = (t - t0)[:, None]
    xp = p.x + p.v * dt + a * dt ** 2 / 2 + j * dt ** 3 / 6
    vp = p.v + a * dt + j * dt ** 2 / 2
    ref = oracle.acc_jerk_pot(p.m, xp, vp, p.eps)
    assert_parity(got, ref, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_energy(kirin_lib, precision):
    p = workloads.config_small()
    with _ctx(p, precision) as k:
        kin, pot = k.energy()
        kin2, pot2 = k.energy(2.0 * p.v)  # velocities given by the caller: K scales by 4, W unchanged
        n_max, tile_i, tile_j = k.query()
    rk, rw = oracle.energy(p.m, p.x, p.v, p.eps)
    assert kin == pytest.approx(rk, rel=1e-13)
    assert pot == pytest.approx(rw, rel=1e-12 if precision == "fp64" else 1e-6)
    assert kin2 == pytest.approx(4.0 * kin, rel=1e-15) and pot2 == pot
    assert n_max >= p.n and tile_i > 0 and tile_j == 128


@pytest.mark.parametrize("precision", PRECISIONS)
def test_device_pointer_twin(kirin_lib, precision):
    import torch
    p = workloads.plummer(3000, 9, eps=0.01)
    dev = torch.device("cuda:0")
    m = torch.tensor(p.m, device=dev)
    x = torch.tensor(p.x, device=dev)
    v = torch.tensor(p.v, device=dev)
    il = torch.tensor(workloads.i_subset(p.n, 1000, 1), device=dev)
    acc = torch.empty((1000, 3), dtype=torch.float64, device=dev)
    jerk = torch.empty_like(acc)
    pot = torch.empty(1000, dtype=torch.float64, device=dev)
    with abi.Kirin(p.n, p.eps, precision=precision, stream=torch.cuda.current_stream().cuda_stream) as k:
        k.set_j_particles_dev(m, x, v)
        k.compute_forces_dev(il, acc, jerk, pot)
        k.sync()
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il.cpu().numpy())
    assert_parity((acc.cpu().numpy(), jerk.cpu().numpy(), pot.cpu().numpy()), ref, precision)


def test_mixed_and_fp64_paths_agree(kirin_lib):
    p = workloads.plummer(4096, 1002, eps=1e-3)
    with _ctx(p, "mixed") as k:
        gm = k.forces()
    with _ctx(p, "fp64") as k:
        gd = k.forces()
    assert_parity(gm, gd, "mixed")


def test_repeated_calls_are_bitwise_reproducible(kirin_lib):
    p = workloads.plummer(5000, 3, eps=0.01)
    il = workloads.i_subset(p.n, 300, 4)
    with _ctx(p, "mixed") as k:
        a = k.forces(il)
        b = k.forces(il)
    for u, w in zip(a, b):
        assert np.array_equal(u, w)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_errors_are_reported_not_crashed(kirin_lib, precision):
    p = workloads.plummer(100, 1, eps=0.01)
    with abi.Kirin(200, p.eps, precision=precision) as k:
        with pytest.raises(abi.KirinError) as e:
            k.compute_forces()
        assert e.value.code == abi.KIRIN_ESTATE
        k.set_j_particles(p.m, p.x, p.v)
        with pytest.raises(abi.KirinError) as e:
            k.compute_forces(np.array([0, 100], dtype=np.int32))
        assert e.value.code == abi.KIRIN_EINVAL
        bad = p.x.copy()
        bad[3, 1] = np.nan
        with pytest.raises(abi.KirinError) as e:
            k.set_j_particles(p.m, bad, p.v)
        assert e.value.code == abi.KIRIN_ENONFINITE
        with pytest.raises(abi.KirinError) as e:
            k.get_acc_jerk_pot()
        assert e.value.code == abi.KIRIN_ESTATE
        with pytest.raises(abi.KirinError) as e:
            k.set_j_particles(p.m, p.x, p.v, first=150)
        assert e.value.code == abi.KIRIN_EINVAL
        # the context is still usable
        got = k.forces()
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps)
    assert_parity(got, ref, precision)


def test_device_side_bad_index_is_flagged(kirin_lib):
    import torch
    p = workloads.plummer(300, 2, eps=0.01)
    dev = torch.device("cuda:0")
    il = torch.tensor([0, 5, 300, 7], dtype=torch.int32, device=dev)  # 300 is out of range
    out = torch.empty((4, 3), dtype=torch.float64, device=dev)
    pot = torch.empty(4, dtype=torch.float64, device=dev)
    with abi.Kirin(p.n, p.eps, stream=torch.cuda.current_stream().cuda_stream) as k:
        k.set_j_particles(p.m, p.x, p.v)
        k.compute_forces_dev(il, out, torch.empty_like(out), pot)
        with pytest.raises(abi.KirinError) as e:
            k.sync()
        assert e.value.code == abi.KIRIN_EINVAL
        k.sync()  # flag cleared, context usable


def test_large_workload_sampled_parity(kirin_lib):
    """N = 2^20, log-normal masses, eps = 4/N, in the bench's launch configuration: full mixed
    evaluations (eps = 4/N, and eps = 0 with r_min = 1e-6) checked on 512 random i against the
    oracle over all j; the FP64 kernel on the same sample."""
    import torch
    from paper_0707_0438_gb300 import autotune
    n = 1 << 20
    p = workloads.config_large(n)
    il = workloads.i_subset(n, 512, seed=77)
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    ref0 = oracle.acc_jerk_pot(p.m, p.x, p.v, 0.0, r_min=1e-6, i_idx=il)
    with abi.Kirin(n, p.eps, precision="mixed") as k:
        k.set_j_particles(p.m, p.x, p.v)
        autotune.install(k, n, torch.cuda.get_device_name(0), "mixed")
        full = k.forces()
        assert_parity(tuple(q[il] for q in full), ref, "mixed", "N=2^20")
        k.set_params(0.0, 1.0, 1e-6, "mixed")
        full0 = k.forces()
        assert_parity(tuple(q[il] for q in full0), ref0, "mixed", "N=2^20 eps=0")
        k.set_params(p.eps, 1.0, 0.0, "fp64")
        assert_parity(k.forces(il), ref, "fp64", "N=2^20 fp64")


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_scaling_by_powers_of_two(kirin_lib, precision):
    """x -> lam x, eps -> lam eps, m -> mu m, v -> nu v with powers of two scale every step of the
    double-single and FP64 arithmetic exactly (lam^2 an even power of two for the reciprocal square
    root): a -> mu a / lam^2, jerk -> mu nu jerk / lam^3, phi -> mu phi / lam, bit for bit, through
    the split reduction of a small block and a full evaluation."""
    p = workloads.plummer(3000, 4242, masses="lognormal", eps=1.0 / 256)
    il = workloads.i_subset(p.n, 77, seed=8)
    lam, mu, nu = 2.0 ** -3, 2.0 ** 5, 2.0 ** 2
    out = []
    for scale in (False, True):
        m, x, v, eps = (mu * p.m, lam * p.x, nu * p.v, lam * p.eps) if scale else (p.m, p.x, p.v, p.eps)
        with abi.Kirin(p.n, eps, precision=precision) as k:
            k.set_j_particles(m, x, v)
            out.append((k.forces(), k.forces(il)))
    for got, ref in zip(out[1], out[0]):
        a, j, f = ref
        assert np.array_equal(got[0], mu / lam ** 2 * a)
        assert np.array_equal(got[1], mu * nu / lam ** 3 * j)
        assert np.array_equal(got[2], mu / lam * f)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_set_nj_shrinks_and_grows_the_j_set(kirin_lib, precision):
    """kirin_set_nj: the force runs over the first n_j particles only (a ragged 3001 of 5000), the full
    set again after growing back, and n_j beyond the highest index ever set is EINVAL."""
    p = workloads.plummer(5000, 515, eps=1.0 / 256)
    nj = 3001
    il = workloads.i_subset(nj, 200, seed=3)
    ref_small = oracle.acc_jerk_pot(p.m[:nj], p.x[:nj], p.v[:nj], p.eps, i_idx=il)
    ref_full = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    with abi.Kirin(6000, p.eps, precision=precision) as k:
        k.set_j_particles(p.m, p.x, p.v)
        k.set_nj(nj)
        assert_parity(k.forces(il), ref_small, precision, "n_j = 3001")
        k.set_nj(p.n)
        assert_parity(k.forces(il), ref_full, precision, "n_j = 5000 again")
        with pytest.raises(abi.KirinError) as e:
            k.set_nj(p.n + 1)
        assert e.value.code == abi.KIRIN_EINVAL


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n", [4096, 65536])
def test_newton_third_law(kirin_lib, precision, n):
    """Sect. 2, Eq. 1: pair forces are equal and opposite, so sum_i m_i a_i = 0 and, differentiating,
    sum_i m_i jerk_i = 0.  The GPU sums each i separately, so the totals vanish only to rounding:
    <= 1e-7 (mixed) and 1e-14 (FP64) of sum_i m_i |a_i| (of sum_i m_i |jerk_i| for the jerk).  A pair
    term whose rounding depends on which particle of the pair is i, or a one-sided bias of the
    reciprocal square root, shows up here."""
    p = workloads.plummer(n, (3003, n), masses="lognormal", eps=1e-3)
    with _ctx(p, precision) as k:
        acc, jerk, _ = k.forces()
    bound = {"mixed": 1e-7, "fp64": 1e-14}[precision]
    for q in (acc, jerk):
        mq = p.m[:, None] * q
        assert np.linalg.norm(mq.sum(axis=0)) <= bound * np.linalg.norm(mq, axis=1).sum()
