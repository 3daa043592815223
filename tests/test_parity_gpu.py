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
    w_cen = None
    if check_central:
        w_cen = Hp.check_central(cen[rows_], res["central"], Hp.central_moment_scale(prob, res["y"], rows_), tol)
    amb = Hp.ambiguous_points(res["y"], res["bins"], prob.n_bins)
    w_h = Hp.check_hist(hs[rows_], res["hist"], Hp.ambiguous_mass(prob, amb, rows_))
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


def _rowblock_3d():
    """A 3-D grid whose middle axis has a multiple of 64 points (the
    tensor-core epilogue's row-block items), first axis not a multiple of the
    16 indices an item takes, a ragged density count, every density kind."""
    rng = np.random.default_rng(77)
    lo, hi = (-3.0, -2.5, -3.1), (3.0, 2.0, 2.9)
    return I.Problem("rowblock3d", (37, 128, 72), lo, hi, I.MODEL_MIXED_3D, (5.0, 0.08),
                     I.random_densities(rng, 300, lo, hi, kinds=(I.GAUSS, I.UNIFORM, I.TRUNCNORM),
                                        sig=(0.3, 0.9), width=(0.5, 1.5)), 300)


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3", "fp32"])
def test_propagate_3d_row_block_items(precision):
    _parity(_rowblock_3d(), precision)


@pytest.mark.parametrize("seed", [211, 212, 213, 214])
def test_propagate_random_ragged_shapes_bf16x3(seed):
    prob = I.random_problem(seed, ndim=2 + seed % 2)
    _parity(prob, "bf16x3")


# ------------------------------------------------- full-size workloads
# The bench's own configurations, run whole on the GPU (the launch
# configuration bench.py times); the oracle computes a seeded set of rows one
# by one: rows 0 and K - 1, one row in every 128-row tile, the rest random.
_FULL = {}


def _full_oracle(name, n_rows):
    """Oracle values (moments, histograms, condition scales) of `n_rows`
    seeded rows of a full-size workload, computed once per module."""
    key = (name, n_rows)
    if key not in _FULL:
        prob = I.config(name)
        rows = Hp.tile_rows(prob.K, n_rows, seed=1000 + int(name[1:]))
        res = O.solve(prob, rows=rows, threads=Hp.oracle_threads())
        res["rows"] = rows
        res["scale"] = Hp.abs_moment_scale(prob, res["y"], rows)
        res["cscale"] = Hp.central_moment_scale(prob, res["y"], rows)
        res["amb"] = Hp.ambiguous_points(res["y"], res["bins"], prob.n_bins)
        _FULL[key] = (prob, res)
    return _FULL[key]


def _full_parity(name, precision, n_rows):
    prob, res = _full_oracle(name, n_rows)
    rows = res["rows"]
    g, raw, cen, hs = gpu_run(prob, precision)
    tol = Hp.TOL[precision]
    Hp.check_moments(raw[rows], res["raw"], res["scale"], tol)
    Hp.check_central(cen[rows], res["central"], res["cscale"], tol)
    amb_mass = Hp.ambiguous_mass(prob, res["amb"], rows)
    Hp.check_hist(hs[rows], res["hist"], amb_mass)
    # every row (not only the oracle's): a probability vector
    assert np.abs(hs.astype(np.float64).sum(axis=1) - 1.0).max() <= 1e-6 + amb_mass
    assert np.isfinite(raw).all() and np.isfinite(cen).all()
    g.close()


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
@pytest.mark.parametrize("name", ["c2", "c3"])
def test_propagate_full_size_1024_rows(name, precision):
    _full_parity(name, precision, 1024)


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_propagate_c4_full_size_512_rows(precision):
    _full_parity("c4", precision, 512)


def test_propagate_c1_full_fp64_all_rows():
    _parity(I.config("c1"), "fp64")


@pytest.mark.parametrize("name", ["c2", "c3", "c4"])
def test_full_size_bins_bit_exact(name):
    """Per-point bin ids of the full-size grids (the cooperative model-and-
    bins kernel with its FP32 screen) against the oracle's exact FP64 rule;
    a point may differ only where the two libms' values straddle an edge.
    The stable sort by bin and the bin offsets are bit-exact."""
    prob = I.config(name)
    vup = vupmod()
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
    g.sync()
    y_g = g.array("y").cpu().numpy()
    b_g = g.array("bins").cpu().numpy()
    y_o = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
    b_o, ymin, ymax = O.bins(y_o, prob.n_bins)
    np.testing.assert_allclose(y_g, y_o, rtol=0, atol=1e-13 * max(1.0, np.abs(y_o).max()))
    # the GPU's bins are exactly the oracle's rule applied to the GPU's values
    b_gy, _, _ = O.bins(y_g, prob.n_bins)
    np.testing.assert_array_equal(b_g, b_gy)
    amb = Hp.ambiguous_points(y_o, b_o, prob.n_bins)
    mism = b_g != b_o
    assert not (mism & ~amb).any(), f"{int((mism & ~amb).sum())} bins differ away from edges"
    info = g.info()
    assert info.ymin == y_g.min() and info.ymax == y_g.max()
    # the model matrix in sorted form (Eq. MUP): the stable sort by bin and
    # the bin offsets, against numpy's stable argsort of the same bins
    p_g = g.array("perm").cpu().numpy()
    off_g = g.array("offsets").cpu().numpy()
    np.testing.assert_array_equal(p_g, np.argsort(b_g, kind="stable"))
    np.testing.assert_array_equal(off_g[:-1], np.searchsorted(np.sort(b_g), np.arange(prob.n_bins)))
    assert off_g[-1] == prob.N
    g.close()


def test_large_output_offset_keeps_central_moments():
    """y = 1000 + sin x1 + 7 sin^2 x2: the power tables are taken about the
    point of the output range nearest 0 (here min y), so the variance of a
    density is not lost to the common offset; raw moments keep their gate."""
    vup = vupmod()
    import torch
    prob = I.config("c2", "small")
    y_o = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi) + 1000.0
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.set_outputs(torch.as_tensor(y_o, device="cuda"), prob.n_bins, 4)
    b_o, _, _ = O.bins(y_o, prob.n_bins)
    res = O.propagate(prob.n, prob.lo, prob.hi, y_o, b_o, prob.n_bins, 4, prob.dens, threads=Hp.oracle_threads())
    rows = np.arange(prob.K)
    zero = np.zeros(y_o.size, np.int32)
    scale = O.propagate(prob.n, prob.lo, prob.hi, np.abs(y_o), zero, 1, 4, prob.dens, threads=Hp.oracle_threads())["raw"]
    c = Hp.shift_point(y_o)
    assert c == y_o.min()
    cscale = O.propagate(prob.n, prob.lo, prob.hi, np.abs(y_o - c), zero, 1, 4, prob.dens,
                         threads=Hp.oracle_threads())["raw"]
    dd = vup.densities_to_device(prob.dens)
    info_checked = False
    for precision in ("fp32", "bf16x3"):
        raw, cen, hs = g.propagate(dd, precision)
        g.sync()
        if not info_checked:
            info = g.info()
            assert info.yshift == c and info.yscale == pytest.approx(y_o.max() - c, rel=1e-15)
            info_checked = True
        tol = Hp.TOL[precision]
        Hp.check_moments(raw.cpu().numpy(), res["raw"], scale, tol)
        Hp.check_central(cen.cpu().numpy(), res["central"], cscale, tol)
        # the variance keeps its relative accuracy where it is not tiny
        var_g, var_o = cen.cpu().numpy()[:, 1], res["central"][:, 1]
        big = var_o > 0.5
        assert big.any()
        assert (np.abs(var_g[big] - var_o[big]) / var_o[big]).max() < 1e3 * tol
        Hp.check_hist(hs.cpu().numpy(), res["hist"])
    g.close()


@pytest.mark.parametrize("form", [-1, 1, 2])
def test_weights_path_matches_oracle(form):
    """The supplied-W path on c2's small grid, each form (automatic choice:
    the sorted block walk; row per lane; general), against the oracle."""
    vup = vupmod()
    import torch
    prob = I.config("c2", "small")
    K = 70
    Wd = np.stack([O.weights(prob.n, prob.lo, prob.hi, prob.dens, k)[0] for k in range(K)])
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    g.set_weights_form(form)
    W = torch.as_tensor(Wd.astype(np.float32), device="cuda")
    raw = torch.empty((K, 4), dtype=torch.float64, device="cuda")
    hist = torch.empty((K, prob.n_bins), dtype=torch.float32, device="cuda")
    vup.vup_propagate_weights(g.h, W, raw, hist)
    g.sync()
    res = O.solve(prob, rows=np.arange(K))
    scale = Hp.abs_moment_scale(prob, res["y"], np.arange(K))
    Hp.check_moments(raw.cpu().numpy(), res["raw"], scale, Hp.TOL["fp32"])
    Hp.check_hist(hist.cpu().numpy(), res["hist"])


@pytest.mark.parametrize("form", [-1, 2])
def test_weights_path_rows_not_16_byte_aligned(form):
    """A grid whose N is not a multiple of 4 (rows of W not 16-byte aligned):
    the automatic choice (the row-per-lane form; the sorted walk's bulk row
    copies need 16-byte rows) and the general form of the supplied-weights
    path, against the oracle."""
    vup = vupmod()
    import torch
    prob = I.Problem("ragged_w", (101, 57), (-2.0, -1.0), (2.5, 1.5), I.MODEL_SIN_SIN2_2D, (1.0, 3.0),
                     I.random_densities(np.random.default_rng(12), 45, (-2.0, -1.0), (2.5, 1.5),
                                        sig=(0.1, 0.8), width=(0.3, 1.0)), 100)
    assert prob.N % 4 != 0
    K = prob.K
    Wd = np.stack([O.weights(prob.n, prob.lo, prob.hi, prob.dens, k)[0] for k in range(K)])
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    g.set_weights_form(form)
    W = torch.as_tensor(Wd.astype(np.float32), device="cuda")
    raw = torch.empty((K, 4), dtype=torch.float64, device="cuda")
    hist = torch.empty((K, prob.n_bins), dtype=torch.float32, device="cuda")
    vup.vup_propagate_weights(g.h, W, raw, hist)
    g.sync()
    res = O.solve(prob, rows=np.arange(K))
    scale = Hp.abs_moment_scale(prob, res["y"], np.arange(K))
    Hp.check_moments(raw.cpu().numpy(), res["raw"], scale, Hp.TOL["fp32"])
    Hp.check_hist(hist.cpu().numpy(), res["hist"])
    with pytest.raises(vup.VUPError):
        g.set_weights_form(3)
    g.close()


def test_weights_path_full_grid_matches_oracle():
    """The supplied-W path on the full c2 grid (1024^2 points, 4096 sorted
    blocks, every CTA over 64 of them) for 48 densities, against the oracle at
    the FP32 gates; a second call reuses the grid's block sort."""
    vup = vupmod()
    import torch
    prob = I.config("c2")
    rows = Hp.tile_rows(prob.K, 48, seed=71)
    Wd = np.stack([O.weights(prob.n, prob.lo, prob.hi, prob.dens, int(k))[0] for k in rows])
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    W = torch.as_tensor(Wd.astype(np.float32), device="cuda")
    del Wd
    res = O.solve(prob, rows=rows, threads=Hp.oracle_threads())
    scale = Hp.abs_moment_scale(prob, res["y"], rows)
    amb = Hp.ambiguous_points(res["y"], res["bins"], prob.n_bins)
    for _ in range(2):
        raw = torch.empty((rows.size, 4), dtype=torch.float64, device="cuda")
        hist = torch.empty((rows.size, prob.n_bins), dtype=torch.float32, device="cuda")
        vup.vup_propagate_weights(g.h, W, raw, hist)
        g.sync()
        Hp.check_moments(raw.cpu().numpy(), res["raw"], scale, Hp.TOL["fp32"])
        Hp.check_hist(hist.cpu().numpy(), res["hist"], Hp.ambiguous_mass(prob, amb, rows))
    g.close()


# ------------------------------------------------------------ IPSA adjoint
# Gradients are gated at tol x their condition scale (oracle ipsa_scale: the
# sum of the absolute values of the products that make up dM_j/dp), the same
# measure as the raw moments' sum W |y|^j.  Var = M2 - M1^2 has the scale
# cond_2 + 2 |M1| cond_1; a central finite difference with h = 1e-3 sigma
# carries a truncation error of (h^2 / 6) times the third derivative, about
# 1.7e-7 of the first (derivatives of a moment under a density of width sigma
# grow by ~1/sigma per order), covered by 1e-6 |fd|.


_IPSA_ORACLE = {}


def _ipsa_oracle(prob, y, rows):
    """Oracle Jacobian and condition scales of `rows`, once per module."""
    key = (prob.name, prob.n, rows.size, int(rows[0]), int(rows[-1]))
    if key not in _IPSA_ORACLE:
        omu, osg = O.ipsa(prob.n, prob.lo, prob.hi, y, 4, prob.dens, rows=rows, threads=Hp.oracle_threads())
        _IPSA_ORACLE[key] = (omu, osg) + Hp.ipsa_condition(prob, y, rows)
    return _IPSA_ORACLE[key]


def _ipsa_case(prob, precision, rows, grad_seed=3):
    vup = vupmod()
    import torch
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    dd = vup.densities_to_device(prob.dens)
    dmu, dsg = g.ipsa(dd, precision)
    g.sync()
    dmu, dsg = dmu.cpu().numpy(), dsg.cpu().numpy()
    y = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
    omu, osg, cmu, csg = _ipsa_oracle(prob, y, rows)
    tol = Hp.TOL[precision]
    Hp.check_ipsa(dmu[rows], omu, cmu, tol, "dM/dmu")
    Hp.check_ipsa(dsg[rows], osg, csg, tol, "dM/dsigma")
    # vector-Jacobian product against the oracle's Jacobian contracted with
    # the same seed: scale sum_j |grad_j| cond_j
    grad = torch.as_tensor(np.random.default_rng(grad_seed).normal(size=(prob.K, 4)), device="cuda")
    vmu, vsg = g.ipsa(dd, precision, grad=grad)
    g.sync()
    gn = grad.cpu().numpy()[rows]
    for got, og, cond in ((vmu, omu, cmu), (vsg, osg, csg)):
        want = np.einsum("kdj,kj->kd", og, gn)
        sc = np.einsum("kdj,kj->kd", cond, np.abs(gn))
        Hp.check_ipsa(got.cpu().numpy()[rows], want, sc, tol, "vjp")
    return g, y, dmu, dsg, cmu, csg


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_ipsa_matches_oracle_and_fd(precision):
    prob = I.config("c4", "small")
    rows = np.arange(0, prob.K, 7)
    g, y, dmu, dsg, cmu, csg = _ipsa_case(prob, precision, rows)
    tol = Hp.TOL[precision]
    # central finite differences of the oracle, h = 1e-3 sigma: dE/dmu, dVar/dsigma
    zero = np.zeros(y.size, np.int32)
    for s in range(3):
        k = rows[s]
        m1 = O.propagate(prob.n, prob.lo, prob.hi, y, zero, 1, 4, prob.dens.take([k]))["raw"][0, 0]
        for d in range(2):
            for which in ("mu", "sigma"):
                h = 1e-3 * prob.dens.sigma[k, d]
                v = []
                for sg_ in (1, -1):
                    dd1 = prob.dens.take([k])
                    getattr(dd1, which)[0, d] += sg_ * h
                    v.append(O.propagate(prob.n, prob.lo, prob.hi, y, zero, 1, 4, dd1)["central"][0])
                fd = (v[0] - v[1]) / (2 * h)
                gpu = (dmu if which == "mu" else dsg)[k, d]
                cond = (cmu if which == "mu" else csg)[s, d]
                gE = gpu[0]
                gVar = gpu[1] - 2 * m1 * gpu[0]
                assert abs(gE - fd[0]) <= tol * cond[0] + 1e-6 * abs(fd[0]), (which, d, gE, fd[0])
                assert abs(gVar - fd[1]) <= tol * (cond[1] + 2 * abs(m1) * cond[0]) + 1e-6 * abs(fd[1]), \
                    (which, d, gVar, fd[1])


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_ipsa_c4_full_size_256_rows(precision):
    """The c4 workload whole (2048^2 grid, K = 65536): the Jacobian and the
    vector-Jacobian product on 256 seeded rows (one in every other 128-row
    tile, rows 0 and K - 1), the launch bench.py times for c4."""
    prob = I.config("c4")
    rows = Hp.tile_rows(prob.K, 256, seed=44, tile=256)
    g, *_ = _ipsa_case(prob, precision, rows)
    g.close()


def _fused_vs_separate(prob, precision, grad_seed=None):
    """vup_propagate_ipsa against vup_propagate + vup_ipsa_sensitivity on the
    same grid and densities: moments, histograms and sensitivities equal."""
    vup = vupmod()
    import torch
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
    dd = vup.densities_to_device(prob.dens)  # kept alive: the struct holds its pointers
    ds = vup.make_densities(dd)
    K, J, B, nd = prob.K, prob.n_moments, prob.n_bins, prob.ndim
    pr = vup.PRECISIONS[precision]
    grad = None
    if grad_seed is not None:
        grad = torch.as_tensor(np.random.default_rng(grad_seed).standard_normal((K, J)), device="cuda")
    shape = (K, nd) if grad is not None else (K, nd, J)

    def outs():
        return (torch.full((K, J), np.nan, dtype=torch.float64, device="cuda"),
                torch.full((K, J), np.nan, dtype=torch.float64, device="cuda"),
                torch.full((K, B), np.nan, dtype=torch.float32, device="cuda"),
                torch.full(shape, np.nan, dtype=torch.float32, device="cuda"),
                torch.full(shape, np.nan, dtype=torch.float32, device="cuda"))
    a, b = outs(), outs()
    vup.vup_propagate(g.h, ds, pr, a[0], a[1], a[2])
    vup.vup_ipsa_sensitivity(g.h, ds, pr, a[3], a[4], grad)
    g.sync()
    vup.vup_propagate_ipsa(g.h, ds, pr, b[0], b[1], b[2], b[3], b[4], grad)
    g.sync()
    for name, x, y in zip(("raw", "central", "hist", "dmu", "dsigma"), a, b):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        assert np.isfinite(y).all(), name
        np.testing.assert_allclose(y, x, rtol=1e-12, atol=1e-300, err_msg=name)
    g.close()


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
@pytest.mark.parametrize("name", ["c2", "c4"])
@pytest.mark.parametrize("vjp", [False, True])
def test_propagate_ipsa_matches_separate_calls(name, precision, vjp):
    _fused_vs_separate(I.config(name, "small"), precision, grad_seed=7 if vjp else None)


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_propagate_ipsa_c4_full_size(precision):
    """The fused call bench.py times for c4 (2048^2, K = 65536) against the two
    separate calls, whose full-size parity with the oracle is tested above."""
    _fused_vs_separate(I.config("c4"), precision, grad_seed=11)


def test_propagate_ipsa_other_grids_run_the_two_calls():
    """Where the fused path does not apply the call runs the two calls in
    turn: a 1-D grid in FP64 gives their results; a 3-D grid reports the
    sensitivities unsupported (as vup_ipsa_sensitivity does) and the TF32
    kinds likewise."""
    vup = vupmod()
    import torch
    prob = I.config("c1", "small")
    _fused_vs_separate(prob, "fp64")
    p3 = I.config("c3", "small")
    g = vup.Grid(p3.n, p3.lo, p3.hi)
    g.eval_model(p3.model_id, p3.theta, p3.n_bins, p3.n_moments)
    dd = vup.densities_to_device(p3.dens)
    ds = vup.make_densities(dd)
    K, J, B = p3.K, p3.n_moments, p3.n_bins
    raw = torch.empty((K, J), dtype=torch.float64, device="cuda")
    cen = torch.empty((K, J), dtype=torch.float64, device="cuda")
    hist = torch.empty((K, B), dtype=torch.float32, device="cuda")
    dmu = torch.empty((K, 3, J), dtype=torch.float32, device="cuda")
    dsg = torch.empty((K, 3, J), dtype=torch.float32, device="cuda")
    with pytest.raises(vup.VUPError) as e:
        vup.vup_propagate_ipsa(g.h, ds, vup.VUP_BF16X3, raw, cen, hist, dmu, dsg)
    assert e.value.status == vup.VUP_ERR_UNSUPPORTED
    g.sync()
    g.close()
    p2 = I.config("c2", "small")
    g = vup.Grid(p2.n, p2.lo, p2.hi)
    g.eval_model(p2.model_id, p2.theta, p2.n_bins, p2.n_moments)
    dd = vup.densities_to_device(p2.dens)
    ds = vup.make_densities(dd)
    K, J, B = p2.K, p2.n_moments, p2.n_bins
    outs = [torch.empty((K, J), dtype=torch.float64, device="cuda") for _ in range(2)] + \
        [torch.empty((K, B), dtype=torch.float32, device="cuda")] + \
        [torch.empty((K, 2, J), dtype=torch.float32, device="cuda") for _ in range(2)]
    with pytest.raises(vup.VUPError) as e:
        vup.vup_propagate_ipsa(g.h, ds, vup.VUP_TF32X3, *outs)
    assert e.value.status == vup.VUP_ERR_UNSUPPORTED
    g.sync()
    g.close()


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
    d0 = vup.densities_to_device(prob.dens.take([]))         # no densities
    with pytest.raises(vup.VUPError) as e:
        g.propagate(d0, "bf16x3")
    assert e.value.status == vup.VUP_ERR_INVALID_ARG
    with pytest.raises(vup.VUPError) as e:
        vup.vup_propagate_weights(g.h, torch.empty((0, prob.N), dtype=torch.float32, device="cuda"))
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
    # the stored values are written with repr (17 significant digits): their
    # own rounding is far below the gate
    cmu, csg = Hp.ipsa_condition(prob, res["y"], np.arange(prob.K))
    Hp.check_ipsa(dmu.cpu().numpy(), stored["dmu"], cmu, Hp.TOL[precision], "dM/dmu")
    Hp.check_ipsa(dsg.cpu().numpy(), stored["dsigma"], csg, Hp.TOL[precision], "dM/dsigma")


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


def test_allocation_failure_returns_oom_and_leaves_outputs_untouched():
    """With the allocation-failure hook armed, a propagation that must grow
    its per-K scratch returns VUP_ERR_OOM before queueing any work (the
    outputs keep their NaN fill); disarmed, the same call succeeds on the same
    grid, and grid creation fails cleanly the same way."""
    vup = vupmod()
    import torch
    prob = I.config("c2", "small")
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    g.propagate(vup.densities_to_device(prob.dens.take(range(10))), "bf16x3")
    g.sync()
    dd = vup.densities_to_device(prob.dens)  # K = 225: more rows than the scratch holds
    K, B = prob.K, prob.n_bins
    raw = torch.full((K, 4), float("nan"), dtype=torch.float64, device="cuda")
    cen = torch.full((K, 4), float("nan"), dtype=torch.float64, device="cuda")
    hist = torch.full((K, B), float("nan"), dtype=torch.float32, device="cuda")
    ds = vup.make_densities(dd)
    vup.vup_debug_fail_alloc(0)
    try:
        with pytest.raises(vup.VUPError) as e:
            vup.vup_propagate(g.h, ds, vup.VUP_BF16X3, raw, cen, hist)
        assert e.value.status == vup.VUP_ERR_OOM
        with pytest.raises(vup.VUPError) as e:
            vup.Grid(prob.n, prob.lo, prob.hi)
        assert e.value.status == vup.VUP_ERR_OOM
    finally:
        vup.vup_debug_fail_alloc(-1)
    g.sync()
    torch.cuda.synchronize()
    assert torch.isnan(raw).all() and torch.isnan(cen).all() and torch.isnan(hist).all()
    vup.vup_propagate(g.h, ds, vup.VUP_BF16X3, raw, cen, hist)
    g.sync()
    res = O.solve(prob, threads=Hp.oracle_threads())
    scale = Hp.abs_moment_scale(prob, res["y"], np.arange(K))
    Hp.check_moments(raw.cpu().numpy(), res["raw"], scale, Hp.TOL["bf16x3"])
    Hp.check_hist(hist.cpu().numpy(), res["hist"])
    g.close()
