"""Coarse-grained IPSA quantities on the GPU (Sec. 5.2, Eq. IPSA, Eq.
IPSAvar) against the FP64 oracle, through the C ABI.

The matrix and field kernels take their decisions (deviation bin, argmax,
interval bounds) in FP64 in the definitions' order, so fed the same inputs
(the GPU's own histogram, range and estimated values) they must agree with
the oracle bit for bit; end to end they are compared with the oracle's own
pipeline within the histogram tolerance."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_11246_gb300 import inputs as I
from tests import helpers as Hp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1908_11246_gb300 import build
    build.build()


def vupmod():
    from paper_1908_11246_gb300 import vup
    return vup


def setup(prob, precision="bf16x3"):
    import torch
    vup = vupmod()
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
    dd = vup.densities_to_device(prob.dens)
    raw, _, hist = g.propagate(dd, precision, central=False)
    centres = dd["mu"].contiguous()
    yref = torch.empty(prob.K, dtype=torch.float64, device="cuda")
    vup.vup_model_at(g.h, centres, yref)
    g.sync()
    return g, raw, hist, yref


CASES = [I.ipsa_example(s, "small") for s in (0.05, 0.5, 3.0)] + [I.config("c2", "small")]


@pytest.mark.parametrize("prob", CASES, ids=[p.name for p in CASES])
def test_estimated_values_match_oracle(prob):
    g, raw, hist, yref = setup(prob)
    ref = O.model_at(prob.model_id, prob.theta, prob.dens.mu)
    np.testing.assert_allclose(yref.cpu().numpy(), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("prob", CASES, ids=[p.name for p in CASES])
@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_deviation_moments_match_oracle_definition(prob, precision):
    """sum W (y - y(l))^j from the GPU raw moments vs the oracle's direct sum,
    within the moment tolerance times the binomial condition scale."""
    import torch
    vup = vupmod()
    g, raw, hist, yref = setup(prob, precision)
    out = torch.empty_like(raw)
    vup.vup_deviation_moments(g.h, raw, yref, out)
    g.sync()
    yr = yref.cpu().numpy()
    res = O.solve(prob)
    D = O.deviation_moments(prob.n, prob.lo, prob.hi, res["y"], prob.n_moments, prob.dens, yr)
    A = np.concatenate([np.ones((prob.K, 1)), Hp.abs_moment_scale(prob, res["y"], np.arange(prob.K))], axis=1)
    from math import comb
    for j in range(1, prob.n_moments + 1):
        scale = sum(comb(j, m) * A[:, m] * np.abs(yr) ** (j - m) for m in range(j + 1))
        err = np.abs(out.cpu().numpy()[:, j - 1] - D[:, j - 1]) / scale
        assert err.max() <= Hp.TOL[precision], (j, err.max())


@pytest.mark.parametrize("prob", CASES, ids=[p.name for p in CASES])
def test_ipsa_matrix_bit_exact_on_same_inputs_and_close_end_to_end(prob):
    import torch
    vup = vupmod()
    g, raw, hist, yref = setup(prob)
    info = g.info()
    span = info.ymax - info.ymin
    nd, dlo, dhi = 2 * prob.n_bins + 3, -span, span
    out = torch.empty((prob.K, nd), dtype=torch.float32, device="cuda")
    vup.vup_ipsa_matrix(g.h, hist, yref, nd, dlo, dhi, out)
    g.sync()
    h = hist.cpu().numpy().astype(np.float64)
    ref = O.ipsa_matrix(h, info.ymin, info.ymax, yref.cpu().numpy(), nd, dlo, dhi)
    np.testing.assert_array_equal(out.cpu().numpy(), ref.astype(np.float32))
    # end to end against the oracle's own histogram, range and estimated values
    res = O.solve(prob)
    yr = O.model_at(prob.model_id, prob.theta, prob.dens.mu)
    ref2 = O.ipsa_matrix(res["hist"], res["y"].min(), res["y"].max(), yr, nd, dlo, dhi)
    m = out.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(m.sum(axis=1), ref2.sum(axis=1), atol=1e-6)
    centres = dlo + (np.arange(nd) + 0.5) * (dhi - dlo) / nd
    np.testing.assert_allclose(m @ centres, ref2 @ centres, atol=1e-5 * span + (dhi - dlo) / nd)


@pytest.mark.parametrize("level", [0.5, 0.9])
def test_sa_fields_bit_exact_on_same_inputs(level):
    import torch
    vup = vupmod()
    prob = I.ipsa_example(0.5, "small")
    g, raw, hist, yref = setup(prob)
    K, B = hist.shape
    rho = torch.rand(K, dtype=torch.float64, device="cuda")
    am = torch.empty(K, dtype=torch.int32, device="cuda")
    ci = torch.empty((K, 2), dtype=torch.int32, device="cuda")
    gl = torch.empty(B, dtype=torch.float64, device="cuda")
    vup.vup_sa_fields(hist, level, rho, am, ci, gl)
    torch.cuda.synchronize()
    a_o, c_o, g_o = O.sa_fields(hist.cpu().numpy().astype(np.float64), level, rho.cpu().numpy())
    np.testing.assert_array_equal(am.cpu().numpy(), a_o)
    np.testing.assert_array_equal(ci.cpu().numpy(), c_o)
    np.testing.assert_allclose(gl.cpu().numpy(), g_o, rtol=1e-13)   # blocked FP64 order
    # uniform weights, global only
    gl2 = torch.empty(B, dtype=torch.float64, device="cuda")
    vup.vup_sa_fields(hist, level, None, None, None, gl2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(gl2.cpu().numpy(), O.sa_fields(hist.cpu().numpy().astype(np.float64), level)[2],
                               rtol=1e-13)


def test_sa_argument_and_state_errors():
    import torch
    vup = vupmod()
    prob = I.ipsa_example(0.5, "small")
    g, raw, hist, yref = setup(prob)
    out = torch.empty((prob.K, 8), dtype=torch.float32, device="cuda")
    for bad in [(8, 1.0, 1.0), (0, -1.0, 1.0), (8, float("nan"), 1.0)]:
        with pytest.raises(vup.VUPError) as e:
            vup.vup_ipsa_matrix(g.h, hist, yref, bad[0], bad[1], bad[2], out)
        assert e.value.status == vup.VUP_ERR_INVALID_ARG
    am = torch.empty(prob.K, dtype=torch.int32, device="cuda")
    for level in (0.0, 1.0):
        with pytest.raises(vup.VUPError) as e:
            vup.vup_sa_fields(hist, level, None, am)
        assert e.value.status == vup.VUP_ERR_INVALID_ARG
    with pytest.raises(vup.VUPError) as e:
        vup.vup_sa_fields(hist, 0.5)
    assert e.value.status == vup.VUP_ERR_INVALID_ARG
    # outputs supplied by the caller: no built-in model to evaluate
    g2 = vup.Grid(prob.n, prob.lo, prob.hi)
    y = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    g2.set_outputs(y, 4)
    x = torch.zeros((3, 2), dtype=torch.float64, device="cuda")
    yy = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(vup.VUPError) as e:
        vup.vup_model_at(g2.h, x, yy)
    assert e.value.status == vup.VUP_ERR_STATE


# ------------------------------------------------------ Bayes-inverted matrix
POST_CASES = [I.config("c2", "small"), I.ipsa_example(0.5, "small"), I.config("c3", "small"),
              I.random_problem(231, ndim=2)]


@pytest.mark.parametrize("prob", POST_CASES, ids=[p.name for p in POST_CASES])
def test_posterior_means_match_oracle(prob):
    import torch
    vup = vupmod()
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
    dd = vup.densities_to_device(prob.dens)
    K, B, nd = prob.K, prob.n_bins, prob.ndim
    hist = torch.empty((K, B), dtype=torch.float32, device="cuda")
    post = torch.empty((K, B, nd), dtype=torch.float32, device="cuda")
    vup.vup_posterior_means(g.h, vup.make_densities(dd), hist, post)
    g.sync()
    res = O.solve(prob)
    ref = O.posterior_means(prob.n, prob.lo, prob.hi, res["bins"], B, prob.dens)
    p, h = post.cpu().numpy().astype(np.float64), hist.cpu().numpy()
    Hp.check_hist(h, res["hist"])
    xmax = np.array([max(abs(prob.lo[d]), abs(prob.hi[d])) for d in range(nd)])
    live = res["hist"] > 1e-9
    err = np.abs(p - ref)[live] / xmax
    assert err.max() <= 2e-5, err.max()
    # law of total expectation against the oracle's direct input means
    xs = O.grid_coords(prob.n, prob.lo, prob.hi)
    mesh = np.meshgrid(*xs, indexing="ij")
    for k in range(0, K, max(1, K // 5)):
        W, _ = O.weights(prob.n, prob.lo, prob.hi, prob.dens, k)
        for d in range(nd):
            assert abs(h[k] @ p[k, :, d] - W @ mesh[d].ravel()) <= 1e-5 * xmax[d]


def test_posterior_means_reject_1d_grids():
    vup = vupmod()
    prob = I.config("c1", "small")
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
    import torch
    dd = vup.densities_to_device(prob.dens)
    post = torch.empty((prob.K, prob.n_bins, 1), dtype=torch.float32, device="cuda")
    with pytest.raises(vup.VUPError) as e:
        vup.vup_posterior_means(g.h, vup.make_densities(dd), None, post)
    assert e.value.status == vup.VUP_ERR_UNSUPPORTED
