"""IPSA through torch.autograd: backward of the VUP moments (hand-written
adjoint kernels) against the FP64 oracle's analytic gradient."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_11246_gb300 import inputs as I
from tests import helpers as Hp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_autograd_backward_matches_oracle(precision):
    import torch

    from paper_1908_11246_gb300 import autograd as AG
    from paper_1908_11246_gb300 import build, vup
    build.build()
    prob = I.config("c4", "small")
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    dd = vup.densities_to_device(prob.dens)
    mu = dd["mu"].clone().requires_grad_(True)
    sg = dd["sigma"].clone().requires_grad_(True)
    raw = AG.VUPMoments.apply(mu, sg, g, dd["kind"], dd["lo"], dd["hi"], precision)
    rng = np.random.default_rng(4)
    a = torch.as_tensor(rng.normal(size=prob.K), device="cuda")
    b = torch.as_tensor(rng.normal(size=prob.K), device="cuda")
    var = raw[:, 1] - raw[:, 0] ** 2
    loss = (a * raw[:, 0] + b * var).sum()
    loss.backward()
    g.sync()
    rows = np.arange(0, prob.K, 11)
    y = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
    omu, osg = O.ipsa(prob.n, prob.lo, prob.hi, y, 4, prob.dens, rows=rows, threads=Hp.oracle_threads())
    fw = O.propagate(prob.n, prob.lo, prob.hi, y, np.zeros(y.size, np.int32), 1, 4, prob.dens, rows=rows)
    M1 = fw["raw"][:, 0]
    an, bn = a.cpu().numpy()[rows], b.cpu().numpy()[rows]
    for got, og in ((mu.grad, omu), (sg.grad, osg)):
        want = an[:, None] * og[:, :, 0] + bn[:, None] * (og[:, :, 1] - 2 * M1[:, None] * og[:, :, 0])
        A = Hp.abs_moment_scale(prob, y, rows)
        scale = 10 * (np.abs(an) * A[:, 0] + np.abs(bn) * 3 * A[:, 1])[:, None] / prob.dens.sigma[rows]
        err = np.abs(got.cpu().numpy()[rows] - want) / scale
        tol = 1e-6 if precision == "fp32" else 2e-5
        assert err.max() <= tol, err.max()
