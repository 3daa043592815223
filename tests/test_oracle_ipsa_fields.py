"""Pins of the oracle's IPSA coarse-grained quantities (Sec. 5.2): the
estimated values y(l), the deviation moments (Delta^2 of Eq. IPSAvar), the
IPSA probability matrix (Eq. IPSA) and the argmax / confidence-interval /
marginalised fields -- each against facts fixed outside the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_11246_gb300 import inputs as I


def gauss(mus, sigmas):
    mus = np.atleast_2d(np.asarray(mus, float))
    sig = np.atleast_2d(np.asarray(sigmas, float))
    K, nd = mus.shape
    return I.Densities(np.zeros((K, nd), np.uint8), mus, sig, np.zeros((K, nd)), np.zeros((K, nd)))


def test_model_at_midpoints_equals_grid_evaluation():
    """The point evaluation and the grid evaluation (pinned by the moment
    closed forms) agree bit for bit at the grid's own midpoints."""
    n, lo, hi = (17, 9), (-5.0, -1.5), (5.0, 1.5)
    y = O.eval_model(I.MODEL_IPSA_EXAMPLE_2D, (), n, lo, hi).reshape(n)
    xs = O.grid_coords(n, lo, hi)
    pts = np.array([[xs[0][a], xs[1][b]] for a in range(n[0]) for b in range(n[1])])
    np.testing.assert_array_equal(O.model_at(I.MODEL_IPSA_EXAMPLE_2D, (), pts), y.ravel())


@pytest.mark.parametrize("a,b,mu,sig", [(2.5, -1.0, 0.3, 0.4), (-0.7, 3.0, -1.1, 0.25)])
def test_deviation_moments_linear_gaussian_closed_form(a, b, mu, sig):
    """y = a x + b, Gaussian at mu, deviations from y(mu): E[dy] = 0,
    Delta^2 = a^2 sigma^2 / 2, E[dy^3] = 0, E[dy^4] = 3 a^4 sigma^4."""
    n, lo, hi = (3000,), (-6.0,), (6.0,)
    y = O.eval_model(I.MODEL_POLY, (b, a, 0.0), n, lo, hi)
    dens = gauss([[mu]], [[sig]])
    yref = O.model_at(I.MODEL_POLY, (b, a, 0.0), [[mu]])
    D = O.deviation_moments(n, lo, hi, y, 4, dens, yref)[0]
    s = abs(a) * sig
    assert abs(D[0]) <= 1e-12 * (1 + abs(a * mu + b))
    assert 0.5 * D[1] == pytest.approx(0.5 * s * s, rel=1e-9)
    assert abs(D[2]) <= 1e-9 * s ** 3
    assert D[3] == pytest.approx(3 * s ** 4, rel=1e-9)


def test_deviation_moments_match_binomial_of_raw_moments():
    """sum W (y - c)^j expanded with the (separately pinned) raw moments."""
    prob = I.config("c2", "small")
    prob.dens = prob.dens.take(range(12))
    res = O.solve(prob)
    yref = np.linspace(-1.0, 5.0, 12)
    D = O.deviation_moments(prob.n, prob.lo, prob.hi, res["y"], 4, prob.dens, yref)
    M = np.concatenate([np.ones((12, 1)), res["raw"]], axis=1)
    from math import comb
    for j in range(1, 5):
        expect = sum(comb(j, m) * M[:, m] * (-yref) ** (j - m) for m in range(j + 1))
        np.testing.assert_allclose(D[:, j - 1], expect, rtol=1e-10, atol=1e-10 * np.abs(yref).max() ** j)


def test_ipsa_matrix_integer_shift_is_exact_translation():
    """With deviation bins as wide as the output bins and an estimated value
    an integer number of bins from ymin, the matrix is the histogram shifted."""
    rng = np.random.default_rng(3)
    K, B = 5, 40
    H = rng.random((K, B))
    H /= H.sum(axis=1, keepdims=True)
    ymin, ymax = -2.0, 8.0                       # w = 0.25
    shifts = rng.integers(0, B, size=K)
    yref = ymin + 0.25 * shifts
    nd = 2 * B
    dlo = -(ymax - ymin)                          # deviation bin e holds c_b - yref with e = b - shift + B
    M = O.ipsa_matrix(H, ymin, ymax, yref, nd, dlo, ymax - ymin)
    for k in range(K):
        expect = np.zeros(nd)
        expect[np.arange(B) - shifts[k] + B] = H[k]
        np.testing.assert_array_equal(M[k], expect)


def test_ipsa_matrix_keeps_mass_and_centres_the_quadratic_example():
    """Every column keeps its mass (clamped edges); for y = x^2 under a
    Gaussian at mu the mean deviation is E[x^2] - mu^2 = sigma^2 within the
    two bin widths' resolution."""
    mu, sig = 0.7, 0.3
    n, lo, hi = (4000,), (-3.0,), (3.0,)
    y = O.eval_model(I.MODEL_POLY, (0.0, 0.0, 1.0), n, lo, hi)
    B = 400
    bins, ymin, ymax = O.bins(y, B)
    dens = gauss([[mu], [0.0]], [[sig], [0.5]])
    H = O.propagate(n, lo, hi, y, bins, B, 2, dens)["hist"]
    yref = O.model_at(I.MODEL_POLY, (0.0, 0.0, 1.0), [[mu], [0.0]])
    nd, dlo, dhi = 300, -3.0, 6.0
    M = O.ipsa_matrix(H, ymin, ymax, yref, nd, dlo, dhi)
    np.testing.assert_allclose(M.sum(axis=1), H.sum(axis=1), rtol=1e-14)
    centres = dlo + (np.arange(nd) + 0.5) * (dhi - dlo) / nd
    w, wd = (ymax - ymin) / B, (dhi - dlo) / nd
    for k, s in enumerate((sig, 0.5)):
        assert abs(M[k] @ centres - s * s) <= w + wd


def test_sa_fields_against_numpy():
    rng = np.random.default_rng(11)
    K, nb = 30, 57
    H = rng.random((K, nb)) ** 3
    H[3] = 0.0
    H[3, 10] = 1.0                               # all mass in one bin
    H[4, [5, 9]] = H[4].max() + 1.0              # a tie: the first index wins
    rho = rng.random(K)
    for level in (0.5, 0.9, 0.99):
        am, ci, g = O.sa_fields(H, level, rho)
        np.testing.assert_array_equal(am, np.argmax(H, axis=1))
        # FP32 sequential sums (the probabilities' own precision)
        Hf = H.astype(np.float32)
        cum = np.cumsum(Hf, axis=1, dtype=np.float32)
        tot = cum[:, -1:]
        lo = np.argmax(cum > np.float32(0.5 * (1 - level)) * tot, axis=1)
        hi = np.argmax(cum >= np.float32(0.5 * (1 + level)) * tot, axis=1)
        np.testing.assert_array_equal(ci[:, 0], lo)
        np.testing.assert_array_equal(ci[:, 1], hi)
        np.testing.assert_allclose(g, rho @ H / rho.sum(), rtol=1e-13)
    _, ci, g = O.sa_fields(H, 0.9)
    np.testing.assert_allclose(g, H.mean(axis=0), rtol=1e-13)
    assert tuple(ci[3]) == (10, 10)


# ------------------------------------------------------ Bayes-inverted matrix
def test_posterior_means_identity_and_monotone_model():
    """sum_b H[b] E[x | b] = E[x] (law of total expectation, exact in the
    discrete setting); for the monotone y = x every posterior mean lies
    inside its bin's x-range."""
    n, lo, hi = (2000,), (-3.0,), (3.0,)
    y = O.eval_model(I.MODEL_POLY, (0.0, 1.0, 0.0), n, lo, hi)
    B = 37
    b, ymin, ymax = O.bins(y, B)
    dens = gauss([[0.4], [-1.0]], [[0.5], [0.8]])
    post = O.posterior_means(n, lo, hi, b, B, dens)
    H = O.propagate(n, lo, hi, y, b, B, 1, dens)["hist"]
    x = O.grid_coords(n, lo, hi)[0]
    for k in range(2):
        W, _ = O.weights(n, lo, hi, dens, k)
        assert H[k] @ post[k, :, 0] == pytest.approx(W @ x, rel=1e-12, abs=1e-13)
        w = (ymax - ymin) / B
        for bb in np.nonzero(H[k] > 0)[0]:
            assert ymin + bb * w - 1e-12 <= post[k, bb, 0] <= ymin + (bb + 1) * w + 1e-12
    assert np.all(post[0, H[0] == 0, :] == 0)


def test_posterior_means_symmetric_square_model():
    """y = x^2 under a Gaussian centred at 0 on a symmetric grid: the two
    preimages +-sqrt(y) carry equal weight, so every posterior mean of x is 0."""
    n, lo, hi = (1000,), (-2.0,), (2.0,)
    y = O.eval_model(I.MODEL_POLY, (0.0, 0.0, 1.0), n, lo, hi)
    b, _, _ = O.bins(y, 25)
    post = O.posterior_means(n, lo, hi, b, 25, gauss([[0.0]], [[0.6]]))
    assert np.abs(post).max() < 1e-12


def test_posterior_means_2d_identity_against_direct_sums():
    prob = I.config("c2", "small")
    prob.dens = prob.dens.take(range(6))
    res = O.solve(prob)
    post = O.posterior_means(prob.n, prob.lo, prob.hi, res["bins"], prob.n_bins, prob.dens)
    xs = O.grid_coords(prob.n, prob.lo, prob.hi)
    X0 = np.repeat(xs[0], prob.n[1])
    X1 = np.tile(xs[1], prob.n[0])
    for k in range(6):
        W, _ = O.weights(prob.n, prob.lo, prob.hi, prob.dens, k)
        for d, X in enumerate((X0, X1)):
            assert res["hist"][k] @ post[k, :, d] == pytest.approx(W @ X, rel=1e-11, abs=1e-12)
            # direct per-bin sums by numpy
            num = np.bincount(res["bins"], weights=W * X, minlength=prob.n_bins)
            den = np.bincount(res["bins"], weights=W, minlength=prob.n_bins)
            expect = np.where(den > 0, num / np.where(den > 0, den, 1), 0.0)
            np.testing.assert_allclose(post[k, :, d], expect, rtol=1e-11, atol=1e-13)
