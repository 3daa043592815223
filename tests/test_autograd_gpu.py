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
    cmu, csg = Hp.ipsa_condition(prob, y, rows)
    fw = O.propagate(prob.n, prob.lo, prob.hi, y, np.zeros(y.size, np.int32), 1, 4, prob.dens, rows=rows)
    M1 = fw["raw"][:, 0]
    A1 = Hp.abs_moment_scale(prob, y, rows)[:, 0]
    an, bn = a.cpu().numpy()[rows], b.cpu().numpy()[rows]
    tol = Hp.TOL[precision]
    # the loss's gradient seed on the raw moments is (a - 2 b M1, b); the
    # GPU's M1 carries tol * A1, which enters through 2 b M1 dM1/dp
    g1, g2 = an - 2 * bn * M1, bn
    for got, og, cond in ((mu.grad, omu, cmu), (sg.grad, osg, csg)):
        want = g1[:, None] * og[:, :, 0] + g2[:, None] * og[:, :, 1]
        scale = (np.abs(g1)[:, None] * cond[:, :, 0] + np.abs(g2)[:, None] * cond[:, :, 1]
                 + 2 * (np.abs(bn) * A1)[:, None] * np.abs(og[:, :, 0]))
        Hp.check_ipsa(got.cpu().numpy()[rows], want, scale, tol, "autograd")
