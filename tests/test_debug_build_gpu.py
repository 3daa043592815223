"""The debug build (libvup_debug.so, compiled with VUP_DEBUG): device bounds
checks on the indices the histogram walks and the supplied-weights walk read
from layouts and sorted words, which record VUP_ERR_BOUNDS instead of
trapping.  On valid inputs every check must pass (no false alarm) and the
results must match the oracle as the release build's do.  No invalid index
is planted on the GPU.

The checks run in a child process with VUP_DEBUG=1 so that the binding loads
the debug library; the release library of this process is untouched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys
sys.path.insert(0, os.path.join(ROOT, "tests"))
sys.path.insert(0, ROOT)
import numpy as np
import torch
import helpers as Hp
from oracle import oracle as O
from paper_1908_11246_gb300 import inputs as I
from paper_1908_11246_gb300 import vup

assert vup.LIB_PATH.endswith("libvup_debug.so"), vup.LIB_PATH
torch.cuda.set_device(0)


def propagate(prob, precision, stream):
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
    if stream is not None:
        g.set_hist_stream(stream)
    raw, cen, hs = g.propagate(vup.densities_to_device(prob.dens), precision)
    g.sync()  # raises VUPError(VUP_ERR_BOUNDS) if a check failed
    out = raw.cpu().numpy(), hs.cpu().numpy()
    g.close()
    return out


# every histogram stream on 2-D (point, interval, record) and the 3-D point
# stream (rest-axis tables in shared memory), against the oracle
for name, streams in (("c2", (None, 0, 1, 2)), ("c3", (None, 0)), ("c4", (None,))):
    prob = I.config(name, "small")
    res = O.solve(prob, threads=Hp.oracle_threads())
    rows = np.arange(prob.K)
    scale = Hp.abs_moment_scale(prob, res["y"], rows)
    amb = Hp.ambiguous_points(res["y"], res["bins"], prob.n_bins)
    amass = Hp.ambiguous_mass(prob, amb, rows)
    for stream in streams:
        raw, hs = propagate(prob, "bf16x3", stream)
        Hp.check_moments(raw, res["raw"], scale, Hp.TOL["bf16x3"])
        Hp.check_hist(hs, res["hist"], amass)
    print(name, "ok", flush=True)

# the supplied-weights walk (sorted blocks, crossing runs)
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
Hp.check_moments(raw.cpu().numpy(), res["raw"], Hp.abs_moment_scale(prob, res["y"], np.arange(K)), Hp.TOL["fp32"])
Hp.check_hist(hist.cpu().numpy(), res["hist"])
g.close()
print("weights ok", flush=True)
"""


@pytest.mark.gpu
def test_debug_build_checks_pass_on_valid_inputs():
    from paper_1908_11246_gb300 import build as B
    so = B.build(debug=True)
    assert so.endswith("libvup_debug.so")
    env = dict(os.environ, VUP_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    for tag in ("c2 ok", "c3 ok", "c4 ok", "weights ok"):
        assert tag in r.stdout, r.stdout
