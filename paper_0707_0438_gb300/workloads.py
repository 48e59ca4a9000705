"""Seeded synthetic inputs shaped like the paper's runs.

This module only draws initial conditions; it holds none of the force,
integrator or energy arithmetic.  Both the CUDA path and the CPU oracle are fed
from here, so that parity tests compare the two on identical arrays.

The paper integrates equal-mass Plummer spheres in N-body (Henon) units,
N = 256 ... 2^20 (Sect. 4, Tables 1-4).  It does not say how the spheres were
drawn; the sampler below is the classic Aarseth, Henon & Wielen (1974) recipe:

* mass fraction X ~ U(0, 0.999) (the 0.999 truncation keeps r finite),
  r = (X^(-2/3) - 1)^(-1/2)                                  (scale a = 1)
* isotropic directions for position and velocity
* speed ratio q by von Neumann rejection on g(q) = q^2 (1 - q^2)^(7/2),
  |v| = q * sqrt(2) * (1 + r^2)^(-1/4)
* scale to Henon units (G = M = 1, E = -1/4 in the continuum limit):
  x *= 3 pi / 16, v *= sqrt(16 / (3 pi))
* move the centre of mass to rest at the origin.

The sample is *not* rescaled to the exact energy of its own N points, since
that would need the potential sum; its energy is -1/4 up to O(N^-1/2) noise.
Every generator takes an explicit seed and uses numpy's PCG64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

HENON_R = 3.0 * math.pi / 16.0
HENON_V = math.sqrt(16.0 / (3.0 * math.pi))


@dataclass
class Particles:
    """A particle set: masses m (n,), positions x (n,3), velocities v (n,3), float64."""

    m: np.ndarray
    x: np.ndarray
    v: np.ndarray
    eps: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.m.shape[0])


def _rng(seed) -> np.random.Generator:
    if isinstance(seed, (tuple, list)):
        seed = [int(s) for s in seed]
    return np.random.Generator(np.random.PCG64(seed))


def _isotropic(rng: np.random.Generator, radius: np.ndarray) -> np.ndarray:
    n = radius.shape[0]
    cos_t = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    out = np.empty((n, 3))
    out[:, 0] = radius * sin_t * np.cos(phi)
    out[:, 1] = radius * sin_t * np.sin(phi)
    out[:, 2] = radius * cos_t
    return out


def plummer(n: int, seed, *, masses: str = "equal", sigma: float = 0.5,
            truncate: float = 0.999, henon: bool = True, eps: float = 0.0) -> Particles:
    """Draw an N-particle Plummer sphere (Aarseth-Henon-Wielen 1974).

    masses = "equal" gives m_i = 1/N; "lognormal" gives m_i proportional to
    exp(sigma * Z_i), Z_i ~ N(0, 1), normalised to a total mass of 1 and drawn
    independently of the positions.  henon=False keeps the a = 1 scale.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = _rng(seed)
    frac = rng.uniform(0.0, truncate, n)
    with np.errstate(divide="ignore"):
        r = np.where(frac > 0.0, (frac ** (-2.0 / 3.0) - 1.0) ** -0.5, 0.0)
    x = _isotropic(rng, r)

    q = np.empty(0)
    while q.shape[0] < n:
        k = max(64, 2 * (n - q.shape[0]))
        qq = rng.uniform(0.0, 1.0, k)
        yy = rng.uniform(0.0, 0.1, k)
        q = np.concatenate([q, qq[yy < qq * qq * (1.0 - qq * qq) ** 3.5]])
    q = q[:n]
    speed = q * math.sqrt(2.0) * (1.0 + r * r) ** -0.25
    v = _isotropic(rng, speed)

    if masses == "equal":
        m = np.full(n, 1.0 / n)
    elif masses == "lognormal":
        w = np.exp(sigma * rng.standard_normal(n))
        m = w / w.sum()
    else:
        raise ValueError(f"unknown mass spectrum {masses!r}")

    if henon:
        x *= HENON_R
        v *= HENON_V
    mt = m.sum()
    x -= (m[:, None] * x).sum(axis=0) / mt
    v -= (m[:, None] * v).sum(axis=0) / mt
    return Particles(np.ascontiguousarray(m), np.ascontiguousarray(x),
                     np.ascontiguousarray(v), eps=eps,
                     meta={"seed": seed, "masses": masses, "henon": henon})


# --- the five workloads (sizes, softening and seeds) -------------------------

def config_small(n: int = 1024) -> Particles:
    """Equal-mass Plummer sphere, eps = 1/256 (the paper's softening, Sect. 4.1), seed 1001."""
    return plummer(n, 1001, eps=1.0 / 256.0)


def config_block(n: int = 65536) -> Particles:
    """Equal-mass Plummer sphere for the block-step Hermite run, eps = 1e-3, seed 1002."""
    return plummer(n, 1002, eps=1.0e-3)


def config_large(n: int = 1 << 20) -> Particles:
    """Log-normal-mass (sigma 0.5) Plummer sphere, eps = 4/N, seed 1003."""
    return plummer(n, 1003, masses="lognormal", sigma=0.5, eps=4.0 / n)


def ensemble_sizes(n_clusters: int = 512, seed: int = 1004, n_lo: int = 256,
                   ratio: float = 64.0) -> np.ndarray:
    """Cluster sizes N_c = floor(n_lo * ratio^U), U ~ U(0,1): log-uniform in [256, 16384)."""
    u = _rng(seed).uniform(0.0, 1.0, n_clusters)
    return np.floor(n_lo * ratio ** u).astype(np.int64)


def ensemble(n_clusters: int = 512, seed: int = 1004, n_lo: int = 256,
             ratio: float = 64.0):
    """Independent equal-mass Plummer clusters, eps_c = 1/N_c; returns (list[Particles], sizes)."""
    sizes = ensemble_sizes(n_clusters, seed, n_lo, ratio)
    out = [plummer(int(nc), (seed, c), eps=1.0 / float(nc)) for c, nc in enumerate(sizes)]
    return out, sizes


def gaussian_cloud(n: int, seed, eps: float) -> Particles:
    """n equal masses (sum 1) at standard-normal positions with velocities 0.1 N(0, 1): a cheap seeded
    set for size and indexing tests far beyond the paper's N (no equilibrium implied)."""
    rng = _rng(seed)
    x = rng.standard_normal((n, 3))
    v = 0.1 * rng.standard_normal((n, 3))
    return Particles(np.full(n, 1.0 / n), x, v, eps=eps, meta={"kind": "gaussian cloud", "seed": seed})


def config_adjoint(n: int = 16384) -> Particles:
    """Equal-mass Plummer sphere for the differentiable leapfrog, eps = 0.01, seed 1005."""
    return plummer(n, 1005, eps=0.01)


def perturb(p: Particles, scale: float = 1.0e-3, seed: int = 1005) -> Particles:
    """Add seeded Gaussian noise of the given scale to positions and velocities."""
    rng = _rng((seed, 7))
    x = p.x + scale * rng.standard_normal(p.x.shape)
    v = p.v + scale * rng.standard_normal(p.v.shape)
    return Particles(p.m.copy(), x, v, eps=p.eps, meta=dict(p.meta, perturbed=scale))


def i_subset(n: int, k: int, seed: int) -> np.ndarray:
    """A seeded, sorted random subset of k distinct indices out of n (int32)."""
    k = min(k, n)
    idx = _rng((seed, 11)).choice(n, size=k, replace=False)
    return np.sort(idx).astype(np.int32)
