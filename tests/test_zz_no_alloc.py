"""The allocation-free supplied-weights entry point against the regular one
and against the FP64 oracle.

vup_propagate_weights_noalloc serves callers that cannot allocate device
memory while running (a fixed memory budget, an allocator that forbids
growth, a host runtime that owns the device heap): its scratch is a fixed
array compiled into the library.  It must give the same moments and
histograms as vup_propagate_weights, call after call (the shared array keeps
the previous call's contents), for every row-group width of its kernel
(bin counts up to 3072, 6144 and 8192 take 8, 4 and 2 rows per CTA) and when
the array's size, not the GPU's width, limits how many point splits it runs;
and it must reject requests larger than that array.
This file is collected last on purpose and is self-contained, so it passes
alone in a fresh process as well as after every other test.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_11246_gb300 import inputs as I
from tests import helpers as Hp

pytestmark = pytest.mark.gpu


def _setup(K, n_bins=256):
    import torch

    from paper_1908_11246_gb300 import build, vup
    build.build()
    prob = I.config("c2", "small")
    prob.n_bins = n_bins
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    Wd = np.stack([O.weights(prob.n, prob.lo, prob.hi, prob.dens, k)[0] for k in range(K)])
    W = torch.as_tensor(Wd.astype(np.float32), device="cuda")
    return vup, torch, prob, g, W


# K = 96 rows: with 4096 and 8192 bins the 16 MiB array holds fewer point
# splits (10 and 5) than the kernel would otherwise run (16)
@pytest.mark.parametrize("n_bins", [256, 4096, 8192])
def test_noalloc_matches_regular_entry_point_and_oracle_twice(n_bins):
    K = 96
    vup, torch, prob, g, W = _setup(K, n_bins)
    B = prob.n_bins
    raw_ref = torch.empty((K, 4), dtype=torch.float64, device="cuda")
    hist_ref = torch.empty((K, B), dtype=torch.float32, device="cuda")
    vup.vup_propagate_weights(g.h, W, raw_ref, hist_ref)
    g.sync()
    rr, hr = raw_ref.cpu().numpy(), hist_ref.cpu().numpy()
    res = O.solve(prob, rows=np.arange(K))
    scale = Hp.abs_moment_scale(prob, res["y"], np.arange(K))
    for call in range(2):
        raw = torch.full((K, 4), float("nan"), dtype=torch.float64, device="cuda")
        hist = torch.full((K, B), float("nan"), dtype=torch.float32, device="cuda")
        # a second call on a different weight scale must not see the first call's partials
        f = 1.0 if call == 0 else 0.5
        vup.vup_propagate_weights_noalloc(g.h, W * f, raw, hist)
        g.sync()
        rn, hn = raw.cpu().numpy(), hist.cpu().numpy()
        Hp.check_moments(rn, rr * f, scale * f, Hp.TOL["fp32"], what="vs regular entry point")
        np.testing.assert_allclose(hn, hr * f, rtol=0, atol=1e-6)
        Hp.check_moments(rn / f, res["raw"], scale, Hp.TOL["fp32"], what="vs oracle")
        Hp.check_hist(hn / f, res["hist"])
    g.close()


def test_noalloc_rejects_requests_beyond_its_array():
    import ctypes as C
    vup, torch, prob, g, W = _setup(4)
    # K * (32 + 4 B) bytes must fit in VUP_STATIC_SCRATCH_BYTES = 16 MiB
    K_big = (16 << 20) // (32 + 4 * prob.n_bins) + 1
    rc = vup.lib().vup_propagate_weights_noalloc(g.h, K_big, C.c_void_p(W.data_ptr()), None, None, None)
    assert rc == vup.VUP_ERR_INVALID_ARG
    g.close()
