"""Shared helpers of the GPU parity tests (CUDA path vs FP64 oracle).

Tolerances (the error measures are stated in the test names):
* bins, sorted order, offsets: bit-exact wherever the oracle's and the GPU's
  model values agree bit for bit; for transcendental models the two libms
  may differ by a few ulp, so a point may change bin only if its oracle value
  lies within that distance of a bin edge.
* raw moments: |M_gpu - M| / sum_i W |y_i|^j  <= 1e-6 (FP32), 2e-5 (BF16x3
  and 3xTF32), 1e-12 (FP64, 1-D).  The denominator is the condition number of the sum.
* central moments: formed in FP64 from the moments of z = (y - c) / s
  (c the point of [ymin, ymax] nearest 0), which amplifies their error by at
  most c_j = (1, 3, 13, 39) times sum W |y - c|^j (Holder bounds).
* IPSA sensitivities: |dM_gpu - dM| <= tol * the sum of the absolute values
  of the products that make up dM_j/dp (oracle ``ipsa_scale``), the same
  measure the raw moments are gated against.
* histograms: |H_gpu - H| <= 1e-6 absolute per bin (+ the mass of points
  whose bin is ambiguous in the sense above, expected 0), and
  |sum_b H - 1| <= 1e-6.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O

TOL = {"fp64": 1e-12, "fp32": 1e-6, "bf16x3": 2e-5, "tf32x3": 2e-5}
CENTRAL_C = np.array([1.0, 3.0, 13.0, 39.0])


def oracle_threads():
    import os
    return os.cpu_count() or 1


def abs_moment_scale(prob, y, rows):
    """sum_i W[k,i] |y_i|^j for j = 1..J from the oracle (moments of |y|)."""
    zero = np.zeros(y.size, np.int32)
    r = O.propagate(prob.n, prob.lo, prob.hi, np.abs(y), zero, 1, prob.n_moments, prob.dens, rows=rows,
                    threads=oracle_threads())
    return r["raw"]


def tile_rows(K, n_rows, seed, tile=128):
    """Seeded distribution rows for full-size parity: 0, K - 1, one row in
    every `tile`-row tile (the tensor-core row tile and the histogram's
    density tile are both 128 rows), then distinct random rows up to n_rows."""
    rng = np.random.default_rng(seed)
    rows = {0, K - 1}
    for t0 in range(0, K, tile):
        rows.add(int(t0 + rng.integers(min(tile, K - t0))))
    n_rows = min(n_rows, K)
    while len(rows) < n_rows:
        rows.update(int(r) for r in rng.choice(K, size=n_rows - len(rows), replace=False))
    return np.array(sorted(rows), np.int64)


def shift_point(y):
    """The point of [min y, max y] nearest 0 (0 when the range holds it): the
    power tables' reference point."""
    ymin, ymax = float(np.min(y)), float(np.max(y))
    return ymin if ymin > 0 else (ymax if ymax < 0 else 0.0)


def central_moment_scale(prob, y, rows):
    """sum_i W[k,i] |y_i - c|^j for j = 1..J (moments of |y - c|)."""
    zero = np.zeros(y.size, np.int32)
    r = O.propagate(prob.n, prob.lo, prob.hi, np.abs(y - shift_point(y)), zero, 1, prob.n_moments, prob.dens,
                    rows=rows, threads=oracle_threads())
    return r["raw"]


def ipsa_condition(prob, y, rows):
    """Condition scales [S, ndim, J] of dM_j/dmu and dM_j/dsigma (oracle)."""
    return O.ipsa_scale(prob.n, prob.lo, prob.hi, y, prob.n_moments, prob.dens, rows=rows,
                        threads=oracle_threads())


def check_ipsa(g_gpu, g_o, cond, tol, what="ipsa"):
    """Gradients against the oracle's analytic ones at tol x condition scale
    (uniform axes: exactly 0 on both sides)."""
    err = np.abs(g_gpu - g_o) / np.maximum(cond, 1e-300)
    worst = float(err.max())
    assert worst <= tol, f"{what}: worst normalised error {worst:.3e} > {tol:.1e} at {np.unravel_index(err.argmax(), err.shape)}"
    return worst


def ambiguous_points(y, bins_o, B, rel=1e-13):
    """Points whose oracle value lies within rel * max|y| of a bin edge."""
    ymin, ymax = y.min(), y.max()
    if ymax == ymin:
        return np.zeros(y.size, bool)
    t = (y - ymin) / (ymax - ymin) * B
    dist = np.abs(t - np.round(t)) * (ymax - ymin) / B
    return dist <= rel * max(1.0, np.abs(y).max())


def ambiguous_mass(prob, amb, rows):
    """Largest probability mass any of `rows` puts on the edge-ambiguous
    points (the oracle's histogram of the 0/1 ambiguity marks), or 0."""
    if not amb.any():
        return 0.0
    y0 = np.zeros(amb.size)
    r = O.propagate(prob.n, prob.lo, prob.hi, y0, amb.astype(np.int32), 2, 1, prob.dens, rows=rows,
                    threads=oracle_threads())
    return float(r["hist"][:, 1].max())


def check_moments(raw_g, raw_o, scale, tol, what="raw"):
    err = np.abs(raw_g - raw_o) / np.maximum(scale, 1e-300)
    worst = float(err.max())
    assert worst <= tol, f"{what}: worst normalised error {worst:.3e} > {tol:.1e} at {np.unravel_index(err.argmax(), err.shape)}"
    return worst


def check_central(cen_g, cen_o, scale, tol):
    J = cen_g.shape[1]
    err = np.abs(cen_g - cen_o) / np.maximum(scale * CENTRAL_C[:J], 1e-300)
    worst = float(err.max())
    assert worst <= tol, f"central: worst {worst:.3e}"
    return worst


def check_hist(h_g, h_o, amb_mass=0.0, tol=1e-6):
    err = np.abs(h_g.astype(np.float64) - h_o)
    worst = float(err.max())
    assert worst <= tol + amb_mass, f"hist: worst abs error {worst:.3e}"
    assert np.abs(h_g.astype(np.float64).sum(axis=1) - 1.0).max() <= 1e-6 + amb_mass
    return worst
