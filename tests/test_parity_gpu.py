"""CUDA path vs FP64 oracle, element by element, on seeded synthetic inputs.

Every call goes through the C ABI (via the ctypes binding).  Sizes are small
enough for the oracle to finish in seconds while spanning several kernel
tiles and ragged tails; the full-size workloads are checked on sampled rows.
"""
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


def gpu_run(prob, precision, moments=True, central=True, hist=True):
    vup = vupmod()
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
    dd = vup.densities_to_device(prob.dens)
    raw, cen, hs = g.propagate(dd, precision, moments, central, hist)
    g.sync()
    f = lambda t: None if t is None else t.cpu().numpy()
    return g, f(raw), f(cen), f(hs)


def exact_model(prob):
    return prob.model_id == I.MODEL_POLY


GRID_CASES = [
    I.config("c1", "small"), I.config("c2", "small"), I.config("c3", "small"), I.config("c4", "small"),
    I.oscillator_batch(5, n_inst=3, side=(40, 90), kk=(10, 30))[1],
    I.Problem("ipsa_ex", (300, 120), (-5.0, -1.5), (5.0, 1.5), I.MODEL_IPSA_EXAMPLE_2D, (),
              I.config("c2", "small").dens, 1000),
    I.Problem("poly3", (17, 33, 65), (-1.0, -2.0, -3.0), (2.0, 1.0, 0.5), I.MODEL_POLY,
              (0.5, 1.0, -0.3, 2.0, 0.1, -1.5, 0.7), I.config("c3", "small").dens, 100),
]


@pytest.mark.parametrize("prob", GRID_CASES, ids=[p.name for p in GRID_CASES])
def test_model_bins_and_sorted_order(prob):
    """y within libm ulp bounds (bit-exact for polynomial models); bins,
    sorted order and bin offsets bit-exact away from edge ties."""
    vup = vupmod()
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
    g.sync()
    y_g = g.array("y").cpu().numpy()
    b_g = g.array("bins").cpu().numpy()
    p_g = g.array("perm").cpu().numpy()
    off_g = g.array("offsets").cpu().numpy()
    y_o = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
    b_o, ymin, ymax = O.bins(y_o, prob.n_bins)
    if exact_model(prob):
        np.testing.assert_array_equal(y_g, y_o)
    else:
        np.testing.assert_allclose(y_g, y_o, rtol=0, atol=1e-13 * max(1.0, np.abs(y_o).max()))
    info = g.info()
    assert info.ymin == y_g.min() and info.ymax == y_g.max()
    amb = Hp.ambiguous_points(y_o, b_o, prob.n_bins)
    mism = b_g != b_o
    assert not (mism & ~amb).any(), f"{int((mism & ~amb).sum())} bins differ away from edges"
    if not mism.any():
        np.testing.assert_array_equal(p_g, np.argsort(b_o, kind="stable"))
        np.testing.assert_array_equal(off_g[:-1], np.searchsorted(np.sort(b_o), np.arange(prob.n_bins)))
        assert off_g[-1] == prob.N
    else:  # still a valid stable sort of the GPU bins
        np.testing.assert_array_equal(p_g, np.argsort(b_g, kind="stable"))


def _parity(prob, precision, rows=None, check_central=True):
    g, raw, cen, hs = gpu_run(prob, precision)
    res = O.solve(prob, rows=rows, threads=Hp.oracle_threads())
    rows_ = np.arange(prob.K) if rows is None else np.asarray(rows)
    tol = Hp.TOL[precision if prob.ndim > 1 else "fp64"]
    scale = Hp.abs_moment_scale(prob, res["y"], rows_)
    w_raw = Hp.check_moments(raw[rows_], res["raw"], scale, tol)
    w_cen = Hp.check_central(cen[rows_], res["central"], scale, tol) if check_central else None
    amb = Hp.ambiguous_points(res["y"], res["bins"], prob.n_bins)
    amb_mass = 0.0
    if amb.any():
        for s, k in enumerate(rows_):
            W, _ = O.weights(prob.n, prob.lo, prob.hi, prob.dens, k)
            amb_mass = max(amb_mass, float(W[amb].sum()))
    w_h = Hp.check_hist(hs[rows_], res["hist"], amb_mass)
    return w_raw, w_cen, w_h


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c4"])
def test_propagate_small_configs_fp32(name):
    prob = I.config(name, "small")
    _parity(prob, "fp64" if name == "c1" else "fp32")


@pytest.mark.parametrize("seed", [201, 202, 203, 204, 205, 206, 207, 208])
def test_propagate_random_ragged_shapes(seed):
    prob = I.random_problem(seed)
    _parity(prob, "fp32")


def test_bf16x3_single_tile():
    """One 128 x 256 tensor-core tile, one 64-wide k-block."""
    prob = I.Problem("tile1", (64, 64), (-2.0, -1.0), (2.0, 1.5), I.MODEL_SIN_SIN2_2D, (1.0, 3.0),
                     I.random_densities(np.random.default_rng(5), 128, (-2.0, -1.0), (2.0, 1.5),
                                        sig=(0.1, 0.8), width=(0.3, 1.0)), 32)
    _parity(prob, "bf16x3")


@pytest.mark.parametrize("name", ["c2", "c3", "c4"])
def test_propagate_small_configs_bf16x3(name):
    _parity(I.config(name, "small"), "bf16x3")


@pytest.mark.parametrize("seed", [211, 212, 213, 214])
def test_propagate_random_ragged_shapes_bf16x3(seed):
    prob = I.random_problem(seed, ndim=2 + seed % 2)
    _parity(prob, "bf16x3")


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_propagate_full_size_sampled_rows_bf16x3(name):
    prob = I.config(name)
    rows = np.random.default_rng(8).choice(prob.K, size=24, replace=False)
    rows = np.concatenate([[0, prob.K - 1], rows])
    _parity(prob, "bf16x3", rows=rows)


def test_propagate_c1_full_fp64_all_rows():
    _parity(I.config("c1"), "fp64")


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_propagate_full_size_sampled_rows_fp32(name):
    prob = I.config(name)
    rows = np.random.default_rng(7).choice(prob.K, size=24, replace=False)
    rows = np.concatenate([[0, prob.K - 1], rows])
    _parity(prob, "fp32", rows=rows)


def test_weights_path_matches_oracle():
    vup = vupmod()
    import torch
    prob = I.config("c2", "small")
    K = 70
    Wd = np.stack([O.weights(prob.n, prob.lo, prob.hi, prob.dens, k)[0] for k in range(K)])
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    W = torch.as_tensor(Wd.astype(np.float32), device="cuda")
    raw = torch.empty((K, 4), dtype=torch.float64, device="cuda")
    hist = torch.empty((K, prob.n_bins), dtype=torch.float32, device="cuda")
    vup.vup_propagate_weights(g.h, W, raw, hist)
    g.sync()
    res = O.solve(prob, rows=np.arange(K))
    scale = Hp.abs_moment_scale(prob, res["y"], np.arange(K))
    Hp.check_moments(raw.cpu().numpy(), res["raw"], scale, 2e-6)
    Hp.check_hist(hist.cpu().numpy(), res["hist"], tol=2e-6)


# ------------------------------------------------------------ IPSA adjoint
def _ipsa_gate(g_gpu, g_or, scale, tol):
    err = np.abs(g_gpu - g_or) / scale
    assert err.max() <= tol, f"worst {err.max():.3e}"
    return float(err.max())


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_ipsa_matches_oracle_and_fd(precision):
    vup = vupmod()
    import torch
    prob = I.config("c4", "small")
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    dd = vup.densities_to_device(prob.dens)
    dmu, dsg = g.ipsa(dd, precision)
    g.sync()
    dmu, dsg = dmu.cpu().numpy(), dsg.cpu().numpy()
    rows = np.arange(0, prob.K, 7)
    y = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
    omu, osg = O.ipsa(prob.n, prob.lo, prob.hi, y, 4, prob.dens, rows=rows, threads=Hp.oracle_threads())
    A = Hp.abs_moment_scale(prob, y, rows)                  # sum W |y|^j
    sig = prob.dens.sigma[rows]                             # [S, ndim]
    scale = 5.0 * A[:, None, :] / sig[:, :, None]
    tol = 1e-6 if precision == "fp32" else 2e-5
    _ipsa_gate(dmu[rows], omu, scale, tol)
    _ipsa_gate(dsg[rows], osg, scale, tol)
    # vector-Jacobian product form equals the contraction of the Jacobian
    grad = torch.as_tensor(np.random.default_rng(3).normal(size=(prob.K, 4)), device="cuda")
    vmu, vsg = g.ipsa(dd, precision, grad=grad)
    g.sync()
    gn = grad.cpu().numpy()
    np.testing.assert_allclose(vmu.cpu().numpy(), np.einsum("kdj,kj->kd", dmu, gn), rtol=1e-4, atol=1e-5 * np.abs(dmu).max())
    np.testing.assert_allclose(vsg.cpu().numpy(), np.einsum("kdj,kj->kd", dsg, gn), rtol=1e-4, atol=1e-5 * np.abs(dsg).max())
    # central finite differences of the oracle, h = 1e-3 sigma: dE/dmu, dVar/dsigma
    zero = np.zeros(y.size, np.int32)
    for s in range(3):
        k = rows[s]
        for d in range(2):
            for which in ("mu", "sigma"):
                h = 1e-3 * prob.dens.sigma[k, d]
                v = []
                for sg_ in (1, -1):
                    dd1 = prob.dens.take([k])
                    getattr(dd1, which)[0, d] += sg_ * h
                    v.append(O.propagate(prob.n, prob.lo, prob.hi, y, zero, 1, 4, dd1)["central"][0])
                fd = (v[0] - v[1]) / (2 * h)
                m1 = O.propagate(prob.n, prob.lo, prob.hi, y, zero, 1, 4, prob.dens.take([k]))["raw"][0, 0]
                gpu = (dmu if which == "mu" else dsg)[k, d]
                gE = gpu[0]
                gVar = gpu[1] - 2 * m1 * gpu[0]
                sc = 5.0 * A[s] / prob.dens.sigma[k, d]
                assert abs(gE - fd[0]) <= tol * sc[0] + 1e-6 * abs(fd[0]), (which, d, gE, fd[0])
                assert abs(gVar - fd[1]) <= 3 * tol * sc[1] + 1e-6 * abs(fd[1]), (which, d, gVar, fd[1])


def test_ipsa_1d_fp64_matches_oracle():
    vup = vupmod()
    prob = I.config("c1", "small")
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    dmu, dsg = g.ipsa(vup.densities_to_device(prob.dens), "fp64")
    g.sync()
    y = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
    omu, osg = O.ipsa(prob.n, prob.lo, prob.hi, y, 4, prob.dens)
    A = Hp.abs_moment_scale(prob, y, np.arange(prob.K))
    sc = A[:, None, :] / prob.dens.sigma[:, :, None]
    assert (np.abs(dmu.cpu().numpy() - omu) / sc).max() < 1e-6
    assert (np.abs(dsg.cpu().numpy() - osg) / sc).max() < 1e-6


# --------------------------------------------------------------- edge cases
def test_single_density_single_bin():
    prob = I.random_problem(301, ndim=2)
    prob.dens = prob.dens.take([0])
    prob.n_bins = 1
    _, raw, cen, hs = gpu_run(prob, "fp32")
    res = O.solve(prob)
    np.testing.assert_allclose(hs, 1.0, atol=1e-6)
    scale = Hp.abs_moment_scale(prob, res["y"], np.arange(1))
    Hp.check_moments(raw, res["raw"], scale, 1e-6)


def test_constant_model_all_mass_in_bin_zero():
    prob = I.Problem("const", (40, 50), (0.0, 0.0), (1.0, 1.0), I.MODEL_POLY, (2.5, 0, 0, 0, 0),
                     I.random_problem(5, ndim=2).dens, 8)
    prob.n, prob.lo, prob.hi = (40, 50), (0.0, 0.0), (1.0, 1.0)
    prob.dens = I.random_densities(np.random.default_rng(1), 33, prob.lo, prob.hi, sig=(0.05, 0.3),
                                   width=(0.1, 0.5))
    _, raw, cen, hs = gpu_run(prob, "fp32")
    np.testing.assert_allclose(hs[:, 0], 1.0, atol=1e-6)
    np.testing.assert_allclose(hs[:, 1:], 0.0, atol=0)
    np.testing.assert_allclose(raw[:, 0], 2.5, rtol=1e-6)
    np.testing.assert_allclose(cen[:, 1], 0.0, atol=1e-5)


def test_empty_support_reported_by_sync():
    vup = vupmod()
    prob = I.random_problem(9, ndim=2, kinds=(I.UNIFORM,))
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    dens = prob.dens.take([0, 1])
    h = (prob.hi[0] - prob.lo[0]) / prob.n[0]
    dens.mu[1, 0] = prob.lo[0] + 2.0 * h     # between midpoints 1 and 2 ...
    dens.sigma[1, 0] = 0.2 * h               # ... and narrower than their gap
    g.propagate(vup.densities_to_device(dens), "fp32")
    with pytest.raises(vup.VUPError) as e:
        g.sync()
    assert e.value.status == vup.VUP_ERR_EMPTY_SUPPORT
    g.sync()  # the condition is cleared once reported


def test_expired_device_wait_reported_by_sync_and_context_survives():
    """A bounded wait that runs out (an mbarrier nothing arrives at) is
    reported as VUP_ERR_TIMEOUT by vup_sync; the next propagation is exact."""
    vup = vupmod()
    prob = I.config("c2", "small")
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
    g.sync()
    vup.vup_selftest_wait(g.h, 2000)
    with pytest.raises(vup.VUPError) as e:
        g.sync()
    assert e.value.status == vup.VUP_ERR_TIMEOUT
    g.sync()  # cleared once reported
    with pytest.raises(vup.VUPError) as e:
        vup.vup_selftest_wait(g.h, 0)
    assert e.value.status == vup.VUP_ERR_INVALID_ARG
    dd = vup.densities_to_device(prob.dens.take(range(64)))
    raw, _, hs = g.propagate(dd, "fp32", central=False)
    g.sync()
    np.testing.assert_allclose(hs.sum(dim=1).cpu().numpy(), 1.0, atol=1e-6)
    assert np.isfinite(raw.cpu().numpy()).all()


def test_state_and_argument_errors():
    vup = vupmod()
    import torch
    prob = I.config("c2", "small")
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    dd = vup.densities_to_device(prob.dens)
    with pytest.raises(vup.VUPError) as e:
        g.propagate(dd, "fp32")
    assert e.value.status == vup.VUP_ERR_STATE
    with pytest.raises(vup.VUPError) as e:
        g.eval_model(I.MODEL_SIN_QUAD_1D, (1, 0.1), 16)      # 1-D model on a 2-D grid
    assert e.value.status == vup.VUP_ERR_INVALID_ARG
    with pytest.raises(vup.VUPError):
        g.eval_model(prob.model_id, prob.theta, 0)            # zero bins
    with pytest.raises(vup.VUPError):
        g.eval_model(prob.model_id, prob.theta, 9000)         # beyond VUP_MAX_BINS
    g.eval_model(prob.model_id, prob.theta, 16)
    with pytest.raises(vup.VUPError) as e:
        g.propagate(dd, "fp64")                               # FP64 only for 1-D grids
    assert e.value.status == vup.VUP_ERR_UNSUPPORTED
    dd3 = vup.densities_to_device(I.config("c3", "small").dens)
    with pytest.raises(vup.VUPError) as e:
        g.propagate(dd3, "fp32")                              # ndim mismatch
    assert e.value.status == vup.VUP_ERR_INVALID_ARG


def test_set_outputs_user_model_matches_builtin():
    vup = vupmod()
    import torch
    prob = I.config("c2", "small")
    y_o = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.set_outputs(torch.as_tensor(y_o, device="cuda"), prob.n_bins, 4)
    raw, cen, hs = g.propagate(vup.densities_to_device(prob.dens), "fp32")
    g.sync()
    res = O.solve(prob)
    scale = Hp.abs_moment_scale(prob, res["y"], np.arange(prob.K))
    Hp.check_moments(raw.cpu().numpy(), res["raw"], scale, 1e-6)
    np.testing.assert_array_equal(g.array("bins").cpu().numpy(), res["bins"])
    Hp.check_hist(hs.cpu().numpy(), res["hist"])


def test_max_bins_and_long_axis():
    prob = I.Problem("maxb", (32767,), (-3.0,), (3.0,), I.MODEL_POLY, (0.0, 1.0, 0.5),
                     I.config("c1", "small").dens.take(range(5)), 8192)
    prob.dens.mu[:, 0] = np.linspace(-2, 2, 5)
    _parity(prob, "fp64")


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_tiny_2d_case_matches_stored_values(precision):
    """The stored oracle values of tests/golden (written by make_golden.py)."""
    from tests.golden import make_golden as G
    prob = [p for p in G.cases() if p.name == "tiny_2d_mixed"][0]
    stored = G.read(prob.name)
    vup = vupmod()
    g, raw, cen, hs = gpu_run(prob, precision)
    res = O.solve(prob)
    scale = Hp.abs_moment_scale(prob, res["y"], np.arange(prob.K))
    Hp.check_moments(raw, stored["raw"], scale, Hp.TOL[precision])
    Hp.check_hist(hs, stored["hist"])
    dmu, dsg = g.ipsa(vup.densities_to_device(prob.dens), precision)
    g.sync()
    sc = np.abs(stored["dmu"]).max() + np.abs(stored["dsigma"]).max()
    assert np.abs(dmu.cpu().numpy() - stored["dmu"]).max() / sc < 10 * Hp.TOL[precision]
    assert np.abs(dsg.cpu().numpy() - stored["dsigma"]).max() / sc < 10 * Hp.TOL[precision]


# ------------------------------------------------------------ TF32 kinds
@pytest.mark.parametrize("name", ["c2", "c3", "c4"])
def test_propagate_small_configs_tf32x3(name):
    """3 x TF32 split products: gated at the BF16x3 tolerance (2e-5)."""
    _parity(I.config(name, "small"), "tf32x3")


@pytest.mark.parametrize("seed", [211, 212])
def test_propagate_random_ragged_shapes_tf32x3(seed):
    prob = I.random_problem(seed, ndim=2 + seed % 2)
    _parity(prob, "tf32x3")


def test_tf32_single_product_is_report_only_accuracy():
    """One TF32 product (10-bit mantissa) is a comparison point: about 1e-3 of
    the condition scale, far from the FP32 gate; histograms are unaffected."""
    prob = I.config("c2", "small")
    g, raw, cen, hs = gpu_run(prob, "tf32")
    res = O.solve(prob)
    scale = Hp.abs_moment_scale(prob, res["y"], np.arange(prob.K))
    err = (np.abs(raw - res["raw"]) / scale).max()
    assert 1e-7 < err < 5e-3, err
    Hp.check_hist(hs, res["hist"])


@pytest.mark.parametrize("prob", [I.config("c2", "small"), I.config("c3", "small"), I.random_problem(411, ndim=2)],
                         ids=["c2", "c3", "ragged2d"])
def test_cooperative_model_bins_match_separate_kernels(prob):
    """A built-in separable model's values, bins and BF16 power table come
    from one cooperative launch; caller-supplied outputs (the same y) take
    the separate range, bins and table kernels.  Bins, moments and histograms
    must be bit-identical (the table bits decide the moments)."""
    vup = vupmod()
    dd = vup.densities_to_device(prob.dens)
    ga = vup.Grid(prob.n, prob.lo, prob.hi)
    ga.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
    ra, _, ha = ga.propagate(dd, "bf16x3", True, False, True)
    ga.sync()
    y = ga.array("y")
    gb = vup.Grid(prob.n, prob.lo, prob.hi)
    gb.set_outputs(y, prob.n_bins, prob.n_moments)
    rb, _, hb = gb.propagate(dd, "bf16x3", True, False, True)
    gb.sync()
    np.testing.assert_array_equal(ga.array("bins").cpu().numpy(), gb.array("bins").cpu().numpy())
    np.testing.assert_array_equal(ra.cpu().numpy(), rb.cpu().numpy())
    np.testing.assert_array_equal(ha.cpu().numpy(), hb.cpu().numpy())
    ga.close()
    gb.close()


def test_profile_timeline_spans_the_streams():
    """vup_profile_timeline: every timed group with its launching stream and
    begin / end times; a propagation that builds its layout uses three streams."""
    vup = vupmod()
    prob = I.config("c2", "small")
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    dd = vup.densities_to_device(prob.dens)
    vup.vup_profile(True)
    try:
        g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
        g.propagate(dd, "bf16x3")
        g.sync()
        tl = vup.vup_profile_timeline()
        agg = vup.vup_profile_read()
    finally:
        vup.vup_profile(False)
    names = {n for n, _, _, _, _ in tl}
    assert {"model_eval", "density_prep", "hist_segmented", "hist_fixup"} <= names
    assert names == set(agg)
    for n, sid, launches, b, e in tl:
        assert 0.0 <= b <= e and launches >= 0
    assert len({sid for _, sid, _, _, _ in tl}) == 3
    g.close()
