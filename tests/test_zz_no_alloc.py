"""The allocation-free supplied-weights entry point against the regular one.

vup_propagate_weights_noalloc serves callers that cannot allocate device
memory while running (a fixed memory budget, an allocator that forbids
growth, a host runtime that owns the device heap): its scratch is a fixed
array compiled into the library.  It must give the same moments and
histograms as vup_propagate_weights, call after call (the shared array keeps
the previous call's contents), and reject requests larger than that array.
This file is collected last on purpose and is self-contained, so it passes
alone in a fresh process as well as after every other test.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_11246_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _setup(K):
    import torch

    from paper_1908_11246_gb300 import build, vup
    build.build()
    prob = I.config("c2", "small")
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, 4)
    Wd = np.stack([O.weights(prob.n, prob.lo, prob.hi, prob.dens, k)[0] for k in range(K)])
    W = torch.as_tensor(Wd.astype(np.float32), device="cuda")
    return vup, torch, prob, g, W


def test_noalloc_matches_regular_entry_point_twice():
    K = 96
    vup, torch, prob, g, W = _setup(K)
    B = prob.n_bins
    raw_ref = torch.empty((K, 4), dtype=torch.float64, device="cuda")
    hist_ref = torch.empty((K, B), dtype=torch.float32, device="cuda")
    vup.vup_propagate_weights(g.h, W, raw_ref, hist_ref)
    g.sync()
    rr, hr = raw_ref.cpu().numpy(), hist_ref.cpu().numpy()
    for call in range(2):
        raw = torch.full((K, 4), float("nan"), dtype=torch.float64, device="cuda")
        hist = torch.full((K, B), float("nan"), dtype=torch.float32, device="cuda")
        # a second call on a different weight scale must not see the first call's partials
        Wc = W if call == 0 else W * 0.5
        vup.vup_propagate_weights_noalloc(g.h, Wc, raw, hist)
        g.sync()
        scale = 1.0 if call == 0 else 0.5
        np.testing.assert_allclose(raw.cpu().numpy(), rr * scale, rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(hist.cpu().numpy(), hr * scale, rtol=0, atol=1e-6)


def test_noalloc_rejects_requests_beyond_its_array():
    import ctypes as C
    vup, torch, prob, g, W = _setup(4)
    # K * (32 + 4 B) bytes must fit in VUP_STATIC_SCRATCH_BYTES = 16 MiB
    K_big = (16 << 20) // (32 + 4 * prob.n_bins) + 1
    rc = vup.lib().vup_propagate_weights_noalloc(g.h, K_big, C.c_void_p(W.data_ptr()), None, None, None)
    assert rc == vup.VUP_ERR_INVALID_ARG
