"""Shared helpers of the GPU parity tests (CUDA path vs FP64 oracle).

Tolerances (the error measures are stated in the test names):
* bins, sorted order, offsets: bit-exact wherever the oracle's and the GPU's
  model values agree bit for bit; for transcendental models the two libms
  may differ by a few ulp, so a point may change bin only if its oracle value
  lies within that distance of a bin edge.
* raw moments: |M_gpu - M| / sum_i W |y_i|^j  <= 1e-6 (FP32), 2e-5 (BF16x3
  and 3xTF32), 1e-12 (FP64, 1-D).  The denominator is the condition number of the sum.
* central moments: the FP64 conversion from raw moments amplifies that
  error by at most c_j = (1, 3, 13, 39) times sum W |y|^j (Holder bounds).
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


def ambiguous_points(y, bins_o, B, rel=1e-13):
    """Points whose oracle value lies within rel * max|y| of a bin edge."""
    ymin, ymax = y.min(), y.max()
    if ymax == ymin:
        return np.zeros(y.size, bool)
    t = (y - ymin) / (ymax - ymin) * B
    dist = np.abs(t - np.round(t)) * (ymax - ymin) / B
    return dist <= rel * max(1.0, np.abs(y).max())


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
