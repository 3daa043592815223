"""Pins of the FP64 oracle to facts fixed by the mathematics, not by the oracle.

Each test targets a different part of the oracle so that a dropped term, a
wrong sign or index, or a transposed operand fails at least one of them:

* closed-form moments of linear / quadratic models under Gaussians
  (midpoint rule on a Gaussian is spectrally exact, Sec. 3);
* the exact discrete moments of a uniform density;
* closed-form truncated-normal moments (bounds on cell edges);
* the additive-separable identity for 2-D product densities;
* a dense one-hot model matrix times the input probability vector via a
  library GEMM (Eq. 5 / Eq. MUP);
* exact rational-arithmetic bin indices (Eq. 4);
* brute-force Monte Carlo (Algorithm "MC - Single probability");
* normalisation invariants;
* IPSA gradients against closed forms and central finite differences.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_11246_gb300 import inputs as I


def gauss_dens(mus, sigmas, kinds=None, lo=None, hi=None):
    mus = np.atleast_2d(np.asarray(mus, float))
    sig = np.atleast_2d(np.asarray(sigmas, float))
    K, nd = mus.shape
    kind = np.zeros((K, nd), np.uint8) if kinds is None else np.asarray(kinds, np.uint8).reshape(K, nd)
    tlo = np.zeros((K, nd)) if lo is None else np.asarray(lo, float).reshape(K, nd)
    thi = np.zeros((K, nd)) if hi is None else np.asarray(hi, float).reshape(K, nd)
    return I.Densities(kind, mus, sig, tlo, thi)


def run(model, theta, n, lo, hi, dens, B=16, J=4):
    y = O.eval_model(model, theta, n, lo, hi)
    b, _, _ = O.bins(y, B)
    return O.propagate(n, lo, hi, y, b, B, J, dens), y, b


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("a,b,mu,sig", [(2.5, -1.0, 0.3, 0.4), (-0.7, 3.0, -1.1, 0.25)])
def test_linear_gaussian_closed_form(a, b, mu, sig):
    # y = b + a x ; E = a mu + b, Var = a^2 s^2, mu3 = 0, mu4 = 3 a^4 s^4
    n, lo, hi = (3000,), (-6.0,), (6.0,)          # h = 0.004, mu +- 8 sigma inside
    out, _, _ = run(I.MODEL_POLY, (b, a, 0.0), n, lo, hi, gauss_dens([[mu]], [[sig]]))
    c = out["central"][0]
    assert c[0] == pytest.approx(a * mu + b, rel=1e-12, abs=1e-12)
    assert c[1] == pytest.approx(a * a * sig * sig, rel=1e-9)
    assert abs(c[2]) <= 1e-9 * abs(a * sig) ** 3
    assert c[3] == pytest.approx(3 * a ** 4 * sig ** 4, rel=1e-9)
    raw = out["raw"][0]
    assert raw[1] == pytest.approx((a * mu + b) ** 2 + a * a * sig * sig, rel=1e-9)


@pytest.mark.parametrize("mu,sig", [(0.4, 0.3), (-1.3, 0.5)])
def test_square_gaussian_closed_form(mu, sig):
    # y = x^2 ; E = mu^2 + s^2, Var = 4 mu^2 s^2 + 2 s^4
    n, lo, hi = (4000,), (-6.0,), (6.0,)
    out, _, _ = run(I.MODEL_POLY, (0.0, 0.0, 1.0), n, lo, hi, gauss_dens([[mu]], [[sig]]))
    c = out["central"][0]
    assert c[0] == pytest.approx(mu * mu + sig * sig, rel=1e-10)
    assert c[1] == pytest.approx(4 * mu * mu * sig * sig + 2 * sig ** 4, rel=1e-9)


def test_product_gaussian_2d_and_3d_closed_form():
    # y = c + sum_d a_d x_d + b_d x_d^2 with independent axes:
    # E = c + sum (a mu + b (mu^2 + s^2)); Var = sum Var_d,
    # Var_d = a^2 s^2 + b^2 (4 mu^2 s^2 + 2 s^4) + 4 a b mu s^2
    for nd in (2, 3):
        n = (260, 300, 240)[:nd]
        lo = (-6.0, -5.0, -7.0)[:nd]
        hi = (6.0, 7.0, 5.0)[:nd]
        mu = np.array([0.3, 1.1, -1.5])[:nd]
        sg = np.array([0.35, 0.45, 0.4])[:nd]
        a = np.array([1.5, -0.5, 0.8])[:nd]
        b = np.array([0.2, 0.7, -0.3])[:nd]
        theta = [0.9]
        for d in range(nd):
            theta += [a[d], b[d]]
        out, _, _ = run(I.MODEL_POLY, theta, n, lo, hi, gauss_dens([mu], [sg]))
        E = 0.9 + np.sum(a * mu + b * (mu * mu + sg * sg))
        V = np.sum(a * a * sg * sg + b * b * (4 * mu * mu * sg * sg + 2 * sg ** 4) + 4 * a * b * mu * sg * sg)
        assert out["central"][0, 0] == pytest.approx(E, rel=1e-10)
        assert out["central"][0, 1] == pytest.approx(V, rel=1e-9)


def test_uniform_discrete_exact():
    # uniform on |x - c| <= w/2: the included midpoints form an arithmetic
    # progression of m points with spacing h; y = x has mean at its centre and
    # variance h^2 (m^2 - 1) / 12 (discrete uniform).
    n, lo, hi = (1000,), (-3.0,), (5.0,)
    h = Fraction(8, 1000)
    c, w = 0.6183, 1.3377
    xs = [Fraction(-3) + (a + Fraction(1, 2)) * h for a in range(n[0])]
    inc = [a for a in range(n[0]) if abs(xs[a] - Fraction(c)) <= Fraction(w) / 2]
    m = len(inc)
    # no midpoint within 1e-9 of the support edge, so the count is unambiguous
    assert all(abs(abs(xs[a] - Fraction(c)) - Fraction(w) / 2) > 1e-9 for a in range(n[0]))
    out, _, _ = run(I.MODEL_POLY, (0.0, 1.0, 0.0), n, lo, hi,
                    gauss_dens([[c]], [[w]], kinds=[[I.UNIFORM]]))
    mean = float((xs[inc[0]] + xs[inc[-1]]) / 2)
    var = float(h * h * (m * m - 1) / 12)
    assert out["central"][0, 0] == pytest.approx(mean, rel=1e-12, abs=1e-12)
    assert out["central"][0, 1] == pytest.approx(var, rel=1e-9)


def _phi(t):
    return math.exp(-0.5 * t * t) / math.sqrt(2 * math.pi)


def _Phi(t):
    return 0.5 * (1 + math.erf(t / math.sqrt(2)))


def test_truncated_normal_closed_form():
    # bounds on cell edges -> midpoint rule over whole cells, O((h/s)^2) error
    n, lo, hi = (4000,), (-10.0,), (10.0,)
    h = 20.0 / 4000
    mu, sg = 0.37, 1.0
    tlo, thi = -10.0 + 1900 * h, -10.0 + 2260 * h   # -0.5 and 1.3
    out, _, _ = run(I.MODEL_POLY, (0.0, 1.0, 0.0), n, lo, hi,
                    gauss_dens([[mu]], [[sg]], kinds=[[I.TRUNCNORM]], lo=[[tlo]], hi=[[thi]]))
    al, be = (tlo - mu) / sg, (thi - mu) / sg
    Zc = _Phi(be) - _Phi(al)
    E = mu + sg * (_phi(al) - _phi(be)) / Zc
    V = sg * sg * (1 + (al * _phi(al) - be * _phi(be)) / Zc - ((_phi(al) - _phi(be)) / Zc) ** 2)
    assert out["central"][0, 0] == pytest.approx(E, rel=2e-6)
    assert out["central"][0, 1] == pytest.approx(V, rel=2e-5)


# ------------------------------------------------------- additive separability
def test_additive_separable_2d_matches_binomial_of_1d():
    # y = g(x1) + h(x2) with a product density: E[y^j] = sum_m C(j,m) E[g^m] E[h^(j-m)]
    n, lo, hi = (150, 170), (-math.pi, -math.pi), (math.pi, math.pi)
    dens = gauss_dens([[0.4, -1.0]], [[0.5, 0.3]])
    J = 4
    out2, _, _ = run(I.MODEL_SIN_SIN2_2D, (1.0, 7.0), n, lo, hi, dens, J=J)
    # 1-D moments via degenerate grids: one axis with a single point
    d1 = gauss_dens([[0.4, 0.0]], [[0.5, 1.0]])
    g, _, _ = run(I.MODEL_SIN_SIN2_2D, (1.0, 0.0), (150, 1), lo, hi, d1, J=J)
    d2 = gauss_dens([[0.0, -1.0]], [[1.0, 0.3]])
    hh, _, _ = run(I.MODEL_SIN_SIN2_2D, (0.0, 7.0), (1, 170), lo, hi, d2, J=J)
    Eg = np.concatenate([[1.0], g["raw"][0]])
    Eh = np.concatenate([[1.0], hh["raw"][0]])
    for j in range(1, J + 1):
        ref = sum(math.comb(j, m) * Eg[m] * Eh[j - m] for m in range(j + 1))
        assert out2["raw"][0, j - 1] == pytest.approx(ref, rel=1e-12)


# ------------------------------------------------------------ library special
def test_dense_model_matrix_gemm_matches_loops():
    # Eq. 5: P(y) = M_{y,x} . P(x) with the one-hot model matrix (Eq. MUP);
    # moments as W @ [y^j].  Tiny inputs, numpy FP64 matmul as the second route.
    prob = I.random_problem(7, ndim=2, max_side=12)
    y = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
    b, _, _ = O.bins(y, prob.n_bins)
    res = O.propagate(prob.n, prob.lo, prob.hi, y, b, prob.n_bins, 4, prob.dens)
    W = np.stack([O.weights(prob.n, prob.lo, prob.hi, prob.dens, k)[0] for k in range(prob.K)])
    Mm = np.zeros((prob.n_bins, y.size))
    Mm[b, np.arange(y.size)] = 1.0
    H = (Mm @ W.T).T
    np.testing.assert_allclose(res["hist"], H, rtol=0, atol=1e-14)
    Y = np.stack([y ** j for j in range(1, 5)], axis=1)
    np.testing.assert_allclose(res["raw"], W @ Y, rtol=1e-13, atol=1e-13)


# -------------------------------------------------------------- exact binning
def test_bins_match_exact_rational_floor():
    rng = np.random.default_rng(11)
    y = np.concatenate([rng.normal(size=4000) * 3.0, [1.25, -7.0, 9.5, 9.5, -7.0]])
    # points exactly on interior edges of 10 bins over [-7, 9.5]
    y = np.concatenate([y, -7.0 + np.arange(1, 10) * 1.65])
    for B in (1, 3, 10, 64, 257):
        b, ymin, ymax = O.bins(y, B)
        assert ymin == y.min() and ymax == y.max()
        lo, rng_ = Fraction(ymin), Fraction(ymax) - Fraction(ymin)
        for i, v in enumerate(y):
            q = (Fraction(v) - lo) * B / rng_
            exact = min(int(math.floor(q)), B - 1)
            if abs(q - round(q)) > Fraction(1, 10 ** 9) or q == B:
                assert b[i] == exact, (B, v)
            else:
                assert abs(int(b[i]) - exact) <= 1
        assert b.min() >= 0 and b.max() <= B - 1
        assert b[np.argmax(y)] == B - 1 and b[np.argmin(y)] == 0


def test_constant_model_single_bin():
    b, ymin, ymax = O.bins(np.full(17, 2.5), 8)
    assert (b == 0).all() and ymin == ymax == 2.5


# ----------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", [101, 102, 103, 104])
def test_normalisation_invariants(seed):
    prob = I.random_problem(seed, max_side={1: 700, 2: 60, 3: 14}[I.random_problem(seed).ndim])
    rows = np.arange(min(prob.K, 12))
    res = O.solve(prob, rows=rows)
    np.testing.assert_allclose(res["wsum"], 1.0, atol=1e-13)
    np.testing.assert_allclose(res["hist"].sum(axis=1), 1.0, atol=1e-13)
    assert (res["hist"] >= 0).all()
    # Jensen / Cauchy-Schwarz: E[y^2] >= E[y]^2; central[0] is the mean
    assert (res["raw"][:, 1] >= res["raw"][:, 0] ** 2 - 1e-12).all()
    np.testing.assert_array_equal(res["central"][:, 0], res["raw"][:, 0])


# --------------------------------------------------------------- Monte Carlo
def _mc_model(model, theta, x):
    if model == I.MODEL_SIN_QUAD_1D:
        return theta[0] * np.sin(x[0]) + theta[1] * x[0] ** 2
    if model == I.MODEL_SIN_SIN2_2D:
        return theta[0] * np.sin(x[0]) + theta[1] * np.sin(x[1]) ** 2
    if model == I.MODEL_MIXED_3D:
        return np.sin(x[0]) + theta[0] * np.sin(x[1]) ** 2 + theta[1] * x[2] ** 4 * np.sin(x[0])
    if model == I.MODEL_OSCILLATOR_2D:
        w, z, T = x[0], x[1], theta[0]
        return np.exp(-z * w * T) * np.cos(w * np.sqrt(1 - z * z) * T)
    if model == I.MODEL_IPSA_EXAMPLE_2D:
        return x[0] ** 2 + 5 * np.sin(3 * x[0]) + x[1]
    raise ValueError


MC_CASES = [
    (I.MODEL_SIN_QUAD_1D, (1.0, 0.1), (4096,), (-5.0,), (5.0,), [0.7], [0.3]),
    (I.MODEL_SIN_SIN2_2D, (1.0, 7.0), (300, 280), (-math.pi,) * 2, (math.pi,) * 2, [0.2, -0.5], [0.3, 0.25]),
    (I.MODEL_MIXED_3D, (7.0, 0.1), (60, 64, 70), (-math.pi,) * 3, (math.pi,) * 3, [0.3, 0.6, -0.4], [0.35, 0.3, 0.35]),
    (I.MODEL_OSCILLATOR_2D, (4.0,), (240, 260), (0.5, 0.01), (5.0, 0.9), [2.0, 0.4], [0.25, 0.05]),
    (I.MODEL_IPSA_EXAMPLE_2D, (), (400, 120), (-5.0, -1.5), (5.0, 1.5), [1.2, 0.0], [0.4, 0.25]),
]


@pytest.mark.parametrize("case", MC_CASES, ids=[f"model{c[0]}" for c in MC_CASES])
def test_monte_carlo_brute_force(case):
    # Algorithm "MC - Single probability": sample the input pdf, evaluate the
    # model, bin.  Means are >= 4 sigma inside the domain and sigma/h >= 4,
    # so the midpoint-rule discretisation error is far below the MC error.
    model, theta, n, lo, hi, mu, sg = case
    nd = len(n)
    rng = np.random.default_rng(1234 + model)
    S = 2_000_000
    x = [rng.normal(mu[d], sg[d], size=S) for d in range(nd)]
    ok = np.ones(S, bool)
    for d in range(nd):
        ok &= (x[d] >= lo[d]) & (x[d] <= hi[d])
    x = [v[ok] for v in x]
    ys = _mc_model(model, theta, x)
    B = 24
    out, y, b = run(model, theta, n, lo, hi, gauss_dens([mu], [sg]), B=B)
    for j in range(1, 5):
        v = ys ** j
        se = v.std() / math.sqrt(v.size)
        assert abs(out["raw"][0, j - 1] - v.mean()) < 5 * se + 1e-12, j
    # histogram: MC frequencies in the oracle's bins; allowance of one grid
    # cell of probability mass per bin edge for the discrete grid
    ymin, ymax = y.min(), y.max()
    t = np.clip(np.floor((ys - ymin) / (ymax - ymin) * B), 0, B - 1).astype(int)
    freq = np.bincount(t, minlength=B) / ys.size
    cell = np.prod([(hi[d] - lo[d]) / n[d] / (sg[d] * math.sqrt(2 * math.pi)) for d in range(nd)])
    edge = 2 * cell * max(n[d] for d in range(nd)) if nd > 1 else 2 * cell
    se = np.sqrt(freq * (1 - freq) / ys.size)
    assert (np.abs(out["hist"][0] - freq) <= 5 * se + edge + 1e-9).all()
    assert np.abs(out["hist"][0] - freq).sum() < 0.05


# ----------------------------------------------------------------------- IPSA
def test_ipsa_closed_forms_linear_and_square():
    n, lo, hi = (4000,), (-6.0,), (6.0,)
    mu, sg = 0.45, 0.35
    y = O.eval_model(I.MODEL_POLY, (0.5, 2.0, 0.0), n, lo, hi)    # y = 0.5 + 2x
    dens = gauss_dens([[mu]], [[sg]])
    dmu, dsg = O.ipsa(n, lo, hi, y, 2, dens)
    fw = O.propagate(n, lo, hi, y, np.zeros(y.size, np.int32), 1, 2, dens)
    M1 = fw["raw"][0, 0]
    assert dmu[0, 0, 0] == pytest.approx(2.0, rel=1e-9)
    dvar = dsg[0, 0, 1] - 2 * M1 * dsg[0, 0, 0]
    assert dvar == pytest.approx(2 * 4.0 * sg, rel=1e-9)         # d(a^2 s^2)/ds
    y2 = O.eval_model(I.MODEL_POLY, (0.0, 0.0, 1.0), n, lo, hi)   # y = x^2
    dmu, dsg = O.ipsa(n, lo, hi, y2, 2, dens)
    fw = O.propagate(n, lo, hi, y2, np.zeros(y2.size, np.int32), 1, 2, dens)
    M1 = fw["raw"][0, 0]
    assert dmu[0, 0, 0] == pytest.approx(2 * mu, rel=1e-9)
    assert dsg[0, 0, 0] == pytest.approx(2 * sg, rel=1e-9)
    dvar = dsg[0, 0, 1] - 2 * M1 * dsg[0, 0, 0]
    assert dvar == pytest.approx(8 * mu * mu * sg + 8 * sg ** 3, rel=1e-9)


def test_ipsa_matches_central_finite_differences():
    # config-4 style model on a small grid, h = 1e-3 sigma
    prob = I.config("c4", "small")
    n = (96, 88)
    rows = [0, 40, 101]
    dens = prob.dens.take(rows)
    y = O.eval_model(prob.model_id, prob.theta, n, prob.lo, prob.hi)
    zb = np.zeros(y.size, np.int32)
    dmu, dsg = O.ipsa(n, prob.lo, prob.hi, y, 4, dens)
    for s in range(len(rows)):
        for d in range(2):
            for which, ref in (("mu", dmu), ("sigma", dsg)):
                h = 1e-3 * dens.sigma[s, d]
                vals = []
                for sgn in (+1, -1):
                    dd = dens.take([s])
                    getattr(dd, which)[0, d] += sgn * h
                    vals.append(O.propagate(n, prob.lo, prob.hi, y, zb, 1, 4, dd)["raw"][0])
                fd = (vals[0] - vals[1]) / (2 * h)
                scale = np.abs(fd).max() + 1e-12
                np.testing.assert_allclose(ref[s, d], fd, rtol=0, atol=1e-6 * scale)


def test_ipsa_uniform_axes_are_zero():
    n, lo, hi = (50, 40), (-1.0, -1.0), (1.0, 1.0)
    y = O.eval_model(I.MODEL_POLY, (0.0, 1.0, 0.0, 1.0, 0.0), n, lo, hi)
    dens = gauss_dens([[0.1, 0.2]], [[0.5, 0.3]], kinds=[[I.UNIFORM, I.GAUSS]])
    dmu, dsg = O.ipsa(n, lo, hi, y, 2, dens)
    assert (dmu[0, 0] == 0).all() and (dsg[0, 0] == 0).all()
    assert dmu[0, 1, 0] != 0


def _abs_normal_moment(p):
    """E|u|^p for a standard normal u: 2^(p/2) Gamma((p+1)/2) / sqrt(pi)."""
    return 2 ** (p / 2) * math.gamma((p + 1) / 2) / math.sqrt(math.pi)


def test_ipsa_scale_closed_forms():
    """Condition scale of dM_j/dmu and dM_j/dsigma (sums of |products|):
    y = a x under a centred Gaussian gives sbar_mu = 0, sbar_sigma = 1/sigma and
    cmu_j = |a sigma|^j E|u|^(j+1) / sigma,
    csg_j = |a sigma|^j (E|u|^(j+2) + E|u|^j) / sigma, u standard normal."""
    sg, a = 0.35, -1.7
    n, lo, hi = (20000,), (-8 * sg,), (8 * sg,)
    y = O.eval_model(I.MODEL_POLY, (0.0, a, 0.0), n, lo, hi)
    cmu, csg = O.ipsa_scale(n, lo, hi, y, 4, gauss_dens([[0.0]], [[sg]]))
    for j in range(1, 5):
        f = abs(a * sg) ** j / sg
        assert cmu[0, 0, j - 1] == pytest.approx(f * _abs_normal_moment(j + 1), rel=1e-4), j
        assert csg[0, 0, j - 1] == pytest.approx(f * (_abs_normal_moment(j + 2) + _abs_normal_moment(j)),
                                                 rel=1e-4), j


def test_ipsa_scale_half_truncated_constant_model():
    """Mean on the domain's lower edge (half the Gaussian truncated away), y = c:
    E s_mu = E|s_mu| = sqrt(2/pi)/sigma, so both terms of cmu count:
    cmu_j = 2 sqrt(2/pi) c^j / sigma; E s_sigma = 1/sigma, csg_j = 2 c^j / sigma."""
    sg, c = 0.4, 1.3
    n, lo, hi = (16000,), (0.0,), (8 * sg,)
    y = O.eval_model(I.MODEL_POLY, (c, 0.0, 0.0), n, lo, hi)
    cmu, csg = O.ipsa_scale(n, lo, hi, y, 3, gauss_dens([[0.0]], [[sg]]))
    for j in range(1, 4):
        assert cmu[0, 0, j - 1] == pytest.approx(2 * math.sqrt(2 / math.pi) * c ** j / sg, rel=1e-4)
        assert csg[0, 0, j - 1] == pytest.approx(2 * c ** j / sg, rel=1e-6)


@pytest.mark.parametrize("seed", [31, 32])
def test_ipsa_scale_bounds_the_sensitivities(seed):
    """Triangle inequality: |dM_j/dp| <= its condition scale, every axis kind."""
    prob = I.random_problem(seed, ndim=2 + seed % 2, max_side=30)
    dens = prob.dens.take(range(min(prob.K, 12)))
    y = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
    dmu, dsg = O.ipsa(prob.n, prob.lo, prob.hi, y, 4, dens)
    cmu, csg = O.ipsa_scale(prob.n, prob.lo, prob.hi, y, 4, dens)
    assert (np.abs(dmu) <= cmu * (1 + 1e-12)).all()
    assert (np.abs(dsg) <= csg * (1 + 1e-12)).all()
    assert (cmu > 0).all() and (csg > 0).all()


def test_empty_support_is_an_error():
    n, lo, hi = (10,), (0.0,), (1.0,)
    y = O.eval_model(I.MODEL_POLY, (0.0, 1.0, 0.0), n, lo, hi)
    # uniform of width 0.02 centred between two midpoints holds no grid point
    dens = gauss_dens([[0.1]], [[0.02]], kinds=[[I.UNIFORM]])
    with pytest.raises(O.OracleError):
        O.propagate(n, lo, hi, y, np.zeros(10, np.int32), 1, 2, dens)
