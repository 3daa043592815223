"""Seeded synthetic workloads shaped like the paper's experiments.

This module only draws parameters (grid extents, density kinds and
parameters, model coefficients).  It performs none of the propagation
arithmetic, so both the CUDA path and the FP64 oracle can consume the
same arrays without sharing any code of the method.

Workload shapes (all synthetic, numpy ``default_rng(seed)``):

* ``c1``  1-D ``y = sin x + 0.1 x^2`` on 4096 midpoints of [-5, 5];
  K = 256 Gaussians, mu ~ U[-4, 4], sigma log-uniform in [0.05, 0.5];
  64 bins, FP64.  (Sec. 4.1 timing experiment, reduced to one axis.)
* ``c2``  2-D ``y = sin x1 + 7 sin^2 x2`` on 1024^2 over [-pi, pi]^2;
  K = 16384 product Gaussians with means on a cell-centred 128 x 128
  lattice of measurement locations, per-axis sigma ~ U[0.02, 0.6];
  256 bins.  (Sec. 4.1 model with unit sine coefficient.)
* ``c3``  3-D ``y = sin x1 + 7 sin^2 x2 + 0.1 x3^4 sin x1`` on 128^3 over
  [-pi, pi]^3; K = 32768; each axis independently Gaussian, uniform
  (width ~ U[0.1, 1]) or truncated normal; 512 bins.
* ``c4``  config-2 model on 2048^2, K = 65536 (256^2 lattice), used with
  the IPSA adjoint.
* ``c5``  512 damped-oscillator instances
  ``y = exp(-zeta w T) cos(w sqrt(1 - zeta^2) T)`` over
  (w, zeta) in [0.5, 5] x [0.01, 0.9], T ~ U[1, 10], square grid side
  log-uniform in [32, 1024], K log-uniform in [64, 8192], 128 bins.

Readings taken where the workload description is silent: means and
uniform centres are drawn inside the domain shrunk by 5 % of its range on
each side (so every support holds grid points); truncated-normal bounds
are ``mu + t_lo sigma`` and ``mu + t_hi sigma`` with t_lo ~ U[-3, -0.5],
t_hi ~ U[0.5, 3]; the lattice of locations is cell-centred.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# density kinds (same numbering as the C ABI)
GAUSS, UNIFORM, TRUNCNORM = 0, 1, 2

# built-in model ids (same numbering as the C ABI)
MODEL_SIN_QUAD_1D = 1      # y = t0 sin x + t1 x^2
MODEL_SIN_SIN2_2D = 2      # y = t0 sin x1 + t1 sin^2 x2
MODEL_MIXED_3D = 3         # y = sin x1 + t0 sin^2 x2 + t1 x3^4 sin x1
MODEL_OSCILLATOR_2D = 4    # y = exp(-x2 x1 t0) cos(x1 sqrt(1 - x2^2) t0)
MODEL_IPSA_EXAMPLE_2D = 5  # y = x1^2 + 5 sin(3 x1) + x2
MODEL_POLY = 6             # y = t0 + sum_d (t[1+2d] x_d + t[2+2d] x_d^2)


@dataclass
class Densities:
    """Structure-of-arrays density parameters, row-major [K][ndim]."""

    kind: np.ndarray   # uint8 [K, ndim]
    mu: np.ndarray     # float64 [K, ndim]  (Gaussian/TN mean, uniform centre)
    sigma: np.ndarray  # float64 [K, ndim]  (Gaussian/TN std, uniform full width)
    lo: np.ndarray     # float64 [K, ndim]  (TN lower bound, absolute)
    hi: np.ndarray     # float64 [K, ndim]  (TN upper bound, absolute)

    @property
    def K(self) -> int:
        return int(self.kind.shape[0])

    @property
    def ndim(self) -> int:
        return int(self.kind.shape[1])

    def take(self, rows) -> "Densities":
        rows = np.asarray(rows, dtype=np.int64)
        return Densities(self.kind[rows].copy(), self.mu[rows].copy(),
                         self.sigma[rows].copy(), self.lo[rows].copy(),
                         self.hi[rows].copy())


@dataclass
class Problem:
    """One VUP instance: grid, model, densities, bins, moments."""

    name: str
    n: tuple            # grid points per axis
    lo: tuple           # domain lower bound per axis
    hi: tuple           # domain upper bound per axis
    model_id: int
    theta: tuple
    dens: Densities
    n_bins: int
    n_moments: int = 4
    precision: str = "fp32"
    extra: dict = field(default_factory=dict)

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    @property
    def K(self) -> int:
        return self.dens.K


def _empty(K, ndim):
    return (np.zeros((K, ndim), np.uint8), np.zeros((K, ndim)), np.ones((K, ndim)),
            np.zeros((K, ndim)), np.zeros((K, ndim)))


def lattice_means(L: int, lo: float, hi: float) -> np.ndarray:
    """Cell-centred lattice of L measurement locations on [lo, hi]."""
    return lo + (np.arange(L) + 0.5) * ((hi - lo) / L)


def gaussian_lattice(rng, L, ndim, lo, hi, sig_lo, sig_hi) -> Densities:
    """Product Gaussians, one per lattice location (k = p1*L + p2 ...)."""
    K = L ** ndim
    kind, mu, sigma, tlo, thi = _empty(K, ndim)
    grids = np.meshgrid(*[lattice_means(L, lo[d], hi[d]) for d in range(ndim)], indexing="ij")
    for d in range(ndim):
        mu[:, d] = grids[d].reshape(-1)
    sigma[:] = rng.uniform(sig_lo, sig_hi, size=(K, ndim))
    return Densities(kind, mu, sigma, tlo, thi)


def random_densities(rng, K, lo, hi, kinds=(GAUSS,), sig=(0.05, 0.6),
                     width=(0.1, 1.0), margin=0.05) -> Densities:
    """Independent per-axis densities with kinds drawn from ``kinds``."""
    ndim = len(lo)
    kind, mu, sigma, tlo, thi = _empty(K, ndim)
    for d in range(ndim):
        R = hi[d] - lo[d]
        kd = rng.choice(np.asarray(kinds, np.uint8), size=K)
        kind[:, d] = kd
        mu[:, d] = rng.uniform(lo[d] + margin * R, hi[d] - margin * R, size=K)
        s = rng.uniform(sig[0], sig[1], size=K)
        w = rng.uniform(width[0], width[1], size=K)
        t_lo = rng.uniform(-3.0, -0.5, size=K)
        t_hi = rng.uniform(0.5, 3.0, size=K)
        sigma[:, d] = np.where(kd == UNIFORM, w, s)
        tlo[:, d] = np.where(kd == TRUNCNORM, mu[:, d] + t_lo * s, 0.0)
        thi[:, d] = np.where(kd == TRUNCNORM, mu[:, d] + t_hi * s, 0.0)
    return Densities(kind, mu, sigma, tlo, thi)


PI = math.pi


def config(name: str, scale: str = "full", seed: int | None = None) -> Problem:
    """Build one of the named workloads.

    ``scale='full'`` gives the published shapes; ``'small'`` keeps the
    model, density recipe and bin count but shrinks grid and K to sizes the
    FP64 oracle handles in seconds while still spanning several kernel tiles
    and a ragged tail.
    """
    small = scale == "small"
    if name == "c1":
        rng = np.random.default_rng(1 if seed is None else seed)
        K = 256 if not small else 37
        N = 4096 if not small else 1000
        kind, mu, sigma, tlo, thi = _empty(K, 1)
        mu[:, 0] = rng.uniform(-4.0, 4.0, size=K)
        sigma[:, 0] = np.exp(rng.uniform(math.log(0.05), math.log(0.5), size=K))
        return Problem("c1", (N,), (-5.0,), (5.0,), MODEL_SIN_QUAD_1D, (1.0, 0.1),
                       Densities(kind, mu, sigma, tlo, thi), 64, 4, "fp64")
    if name in ("c2", "c4"):
        is4 = name == "c4"
        rng = np.random.default_rng((4 if is4 else 2) if seed is None else seed)
        if small:
            n = (200, 328) if not is4 else (264, 136)
            L = 15 if not is4 else 13
        else:
            n = (1024, 1024) if not is4 else (2048, 2048)
            L = 128 if not is4 else 256
        dens = gaussian_lattice(rng, L, 2, (-PI, -PI), (PI, PI), 0.02, 0.6)
        return Problem(name, n, (-PI, -PI), (PI, PI), MODEL_SIN_SIN2_2D, (1.0, 7.0),
                       dens, 256, 4, "bf16x3")
    if name == "c3":
        rng = np.random.default_rng(3 if seed is None else seed)
        n = (128, 128, 128) if not small else (24, 40, 72)
        K = 32768 if not small else 300
        lo, hi = (-PI,) * 3, (PI,) * 3
        # the coarse small grid (h up to 0.26) keeps every support non-empty
        # with widths and sigmas of at least 1.3 h
        sig, width = ((0.05, 0.6), (0.1, 1.0)) if not small else ((0.35, 0.6), (0.35, 1.0))
        dens = random_densities(rng, K, lo, hi, kinds=(GAUSS, UNIFORM, TRUNCNORM), sig=sig,
                                width=width)
        return Problem("c3", n, lo, hi, MODEL_MIXED_3D, (7.0, 0.1), dens, 512, 4, "bf16x3")
    if name == "ipsa":
        return ipsa_example(0.5, scale)
    raise ValueError(name)


def ipsa_example(sigma_l: float = 0.5, scale: str = "full") -> Problem:
    """The IPSA example of Sec. 5.3: y = x^2 + 5 sin(3x) + alpha on a
    1000 x 1000 midpoint grid over [-5, 5] x [-1.5, 1.5], L = 1000
    measurement locations l (cell-centred over [-5, 5]) with Gaussian
    measurement uncertainty sigma_l on x and alpha ~ N(0, 0.25^2); 1000 bins.
    The alpha range (+-6 sigma_alpha) and the x grid extent are readings of
    the text, which states neither."""
    small = scale == "small"
    n = (300, 120) if small else (1000, 1000)
    L = 37 if small else 1000
    kind, mu, sigma, tlo, thi = _empty(L, 2)
    mu[:, 0] = lattice_means(L, -5.0, 5.0)
    sigma[:, 0] = sigma_l
    mu[:, 1] = 0.0
    sigma[:, 1] = 0.25
    return Problem(f"ipsa_s{sigma_l:g}", n, (-5.0, -1.5), (5.0, 1.5), MODEL_IPSA_EXAMPLE_2D, (),
                   Densities(kind, mu, sigma, tlo, thi), 100 if small else 1000, 4, "bf16x3")


def oscillator_batch(seed: int = 5, n_inst: int = 512, side=(32, 1024), kk=(64, 8192),
                     n_bins: int = 128) -> list[Problem]:
    """Config-5 style batch of uneven damped-oscillator instances."""
    rng = np.random.default_rng(seed)
    lo, hi = (0.5, 0.01), (5.0, 0.9)
    out = []
    for i in range(n_inst):
        s = int(round(math.exp(rng.uniform(math.log(side[0]), math.log(side[1])))))
        K = int(round(math.exp(rng.uniform(math.log(kk[0]), math.log(kk[1])))))
        T = float(rng.uniform(1.0, 10.0))
        kind, mu, sigma, tlo, thi = _empty(K, 2)
        for d in range(2):
            R = hi[d] - lo[d]
            mu[:, d] = rng.uniform(lo[d] + 0.05 * R, hi[d] - 0.05 * R, size=K)
            sigma[:, d] = rng.uniform(0.02, 0.2, size=K) * R
        out.append(Problem(f"c5_{i}", (s, s), lo, hi, MODEL_OSCILLATOR_2D, (T,),
                           Densities(kind, mu, sigma, tlo, thi), n_bins, 4, "bf16x3"))
    return out


def random_problem(seed: int, ndim: int | None = None, kinds=(GAUSS, UNIFORM, TRUNCNORM),
                   max_side: int | None = None) -> Problem:
    """Randomised small shape (ragged sizes) for parity sweeps."""
    rng = np.random.default_rng(seed)
    if ndim is None:
        ndim = int(rng.integers(1, 4))
    if max_side is None:
        max_side = {1: 3000, 2: 300, 3: 56}[ndim]
    n = tuple(int(rng.integers(5, max_side + 1)) for _ in range(ndim))
    lo = tuple(float(rng.uniform(-4, 0)) for _ in range(ndim))
    hi = tuple(float(lo[d] + rng.uniform(1.0, 8.0)) for d in range(ndim))
    K = int(rng.integers(1, 260))
    if ndim == 1:
        model, theta = MODEL_SIN_QUAD_1D, (float(rng.uniform(0.5, 2)), float(rng.uniform(-0.3, 0.3)))
    elif ndim == 2:
        model, theta = MODEL_SIN_SIN2_2D, (float(rng.uniform(0.5, 2)), float(rng.uniform(1, 8)))
    else:
        model, theta = MODEL_MIXED_3D, (float(rng.uniform(1, 8)), float(rng.uniform(0.01, 0.2)))
    # widths scaled to the domain so supports always hold grid points
    span = min(hi[d] - lo[d] for d in range(ndim))
    hmax = max((hi[d] - lo[d]) / n[d] for d in range(ndim))
    s_lo = max(0.02 * span, 1.5 * hmax)
    w_lo = max(0.05 * span, 3.0 * hmax)
    sig = (s_lo, max(1.5 * s_lo, 0.3 * span))
    width = (w_lo, max(1.5 * w_lo, 0.4 * span))
    dens = random_densities(rng, K, lo, hi, kinds=kinds, sig=sig, width=width, margin=0.1)
    B = int(rng.choice([1, 2, 7, 64, 100, 256, 513]))
    return Problem(f"rand{seed}", n, lo, hi, model, theta, dens, B, 4, "fp32")
