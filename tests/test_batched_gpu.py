"""Batched uneven propagation (many independent 2-D instances per call) vs
the per-instance path and the FP64 oracle.

The batch mixes damped-oscillator instances of uneven grid sides and density
counts with random 2-D problems (every density kind, bin counts from 1 to
513); all calls go through the C ABI.
"""
import json
import os
import tempfile

import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_11246_gb300 import inputs as I
from tests import helpers as Hp

pytestmark = pytest.mark.gpu

# the library reads this at its first batched call in the process
_TUNE_FILE = os.path.join(tempfile.mkdtemp(prefix="vup_tune_"), "tune.jsonl")
os.environ["VUP_TUNE_CACHE"] = _TUNE_FILE


def vupmod():
    from paper_1908_11246_gb300 import vup
    return vup


def batch_problems():
    probs = I.oscillator_batch(7, n_inst=10, side=(16, 160), kk=(3, 200), n_bins=128)
    for seed in (401, 402, 403, 404, 405, 406):
        probs.append(I.random_problem(seed, ndim=2))
    return probs


@pytest.fixture(scope="module")
def batch():
    from paper_1908_11246_gb300 import build
    build.build()
    vup = vupmod()
    probs = batch_problems()
    grids, dens = [], []
    for p in probs:
        g = vup.Grid(p.n, p.lo, p.hi)
        g.eval_model(p.model_id, p.theta, p.n_bins, p.n_moments)
        grids.append(g)
        dens.append(vup.densities_to_device(p.dens))
    oracle = [O.solve(p, threads=Hp.oracle_threads()) for p in probs]
    return probs, grids, dens, oracle


def _host(ts):
    return [None if t is None else t.cpu().numpy() for t in ts]


def _sync(grids):
    import torch
    torch.cuda.synchronize()
    for g in grids:
        g.sync()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_batched_matches_oracle(batch, precision):
    vup = vupmod()
    probs, grids, dens, oracle = batch
    raws, hists = vup.propagate_batched(grids, dens, precision)
    _sync(grids)
    for p, r, h, res in zip(probs, _host(raws), _host(hists), oracle):
        rows = np.arange(p.K)
        scale = Hp.abs_moment_scale(p, res["y"], rows)
        Hp.check_moments(r, res["raw"], scale, Hp.TOL[precision], what=p.name)
        amb = Hp.ambiguous_points(res["y"], res["bins"], p.n_bins)
        Hp.check_hist(h, res["hist"], Hp.ambiguous_mass(p, amb, rows))


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_batched_matches_single_instance_path(batch, precision):
    """Histograms and FP32 moments are the same arithmetic in the same order
    as the one-instance path (bit-identical); BF16x3 moments may use narrower
    tensor-core tiles, so they agree within the BF16x3 tolerance."""
    vup = vupmod()
    probs, grids, dens, oracle = batch
    raws, hists = vup.propagate_batched(grids, dens, precision)
    _sync(grids)
    raws, hists = _host(raws), _host(hists)
    for i, (p, g, dd) in enumerate(zip(probs, grids, dens)):
        r1, _, h1 = g.propagate(dd, precision, central=False)
        g.sync()
        r1, h1 = r1.cpu().numpy(), h1.cpu().numpy()
        np.testing.assert_array_equal(hists[i], h1, err_msg=p.name)
        if precision == "fp32":
            np.testing.assert_array_equal(raws[i], r1, err_msg=p.name)
        else:
            scale = Hp.abs_moment_scale(p, oracle[i]["y"], np.arange(p.K))
            Hp.check_moments(raws[i], r1, scale, 2 * Hp.TOL["bf16x3"], what=p.name)


def test_second_call_replays_graph(batch):
    vup = vupmod()
    probs, grids, dens, _ = batch
    out = vup.batched_outputs(grids, dens)
    vup.propagate_batched(grids, dens, "bf16x3", out=out)
    _sync(grids)
    first = [_host(out[0]), _host(out[1])]
    # (the caching allocator may hand back an earlier call's output addresses,
    # in which case even this call replays a remembered graph)
    assert vup.vup_batched_report()["source"] in (0, 1, 2)
    for t in out[0] + out[1]:
        t.fill_(-1)
    vup.propagate_batched(grids, dens, "bf16x3", out=out)
    _sync(grids)
    rep = vup.vup_batched_report()
    assert rep["source"] == 0 and rep["bn_cap"] in (64, 128, 256)
    for a, b in zip(first[0] + first[1], _host(out[0]) + _host(out[1])):
        np.testing.assert_array_equal(a, b)


def test_tuner_times_new_shapes_and_records_them(batch):
    vup = vupmod()
    probs, grids, dens, oracle = batch
    sub = [0, 3, 5, 11, 14]
    g_sub, d_sub = [grids[i] for i in sub], [dens[i] for i in sub]
    before = open(_TUNE_FILE).read().splitlines() if os.path.exists(_TUNE_FILE) else []
    raws, hists = vup.propagate_batched(g_sub, d_sub, "bf16x3")
    _sync(g_sub)
    rep = vup.vup_batched_report()
    assert rep["source"] == 2 and rep["tune_ms"] > 0
    lines = open(_TUNE_FILE).read().splitlines()
    assert len(lines) == len(before) + 1
    rec = json.loads(lines[-1])
    assert rec["bn_cap"] == rep["bn_cap"] and set(rec["ms"]) == {"256", "128", "64"}
    assert rec["bn_cap"] == int(min(rec["ms"], key=rec["ms"].get))
    # the same shape with other output buffers reuses the decision without timing
    keep = (raws, hists)
    vup.propagate_batched(g_sub, d_sub, "bf16x3")
    _sync(g_sub)
    del keep
    rep2 = vup.vup_batched_report()
    assert rep2["source"] == 1 and rep2["bn_cap"] == rep["bn_cap"] and rep2["tune_ms"] == 0
    for i, r in zip(sub, _host(raws)):
        p = probs[i]
        scale = Hp.abs_moment_scale(p, oracle[i]["y"], np.arange(p.K))
        Hp.check_moments(r, oracle[i]["raw"], scale, Hp.TOL["bf16x3"], what=p.name)


def test_capture_into_caller_graph(batch):
    import torch
    vup = vupmod()
    probs, grids, dens, _ = batch
    out = vup.batched_outputs(grids, dens)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    vup.propagate_batched(grids, dens, "fp32", out=out, stream=s)   # builds the plan
    s.synchronize()
    ref = _host(out[0]) + _host(out[1])
    for t in out[0] + out[1]:
        t.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        vup.propagate_batched(grids, dens, "fp32", out=out, stream=s)
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(ref, _host(out[0]) + _host(out[1])):
        np.testing.assert_array_equal(a, b)


def test_profiled_call_times_each_stage(batch):
    vup = vupmod()
    probs, grids, dens, _ = batch
    out = vup.batched_outputs(grids, dens)
    vup.propagate_batched(grids, dens, "bf16x3", out=out)
    vup.vup_profile(True)
    try:
        vup.propagate_batched(grids, dens, "bf16x3", out=out)
        _sync(grids)
        prof = vup.vup_profile_read()
    finally:
        vup.vup_profile(False)
    for name in ("density_prep_batched", "moments_bf16x3_tc_batched", "moments_finish_fp64_batched",
                 "hist_segmented_batched"):
        assert name in prof, sorted(prof)


def test_batched_argument_errors(batch):
    vup = vupmod()
    probs, grids, dens, _ = batch
    # FP64 is the 1-D path only
    with pytest.raises(vup.VUPError) as e:
        vup.propagate_batched(grids[:2], dens[:2], "fp64")
    assert e.value.status == vup.VUP_ERR_UNSUPPORTED
    # a 3-D grid is not batched
    p3 = I.random_problem(7, ndim=3, max_side=20)
    g3 = vup.Grid(p3.n, p3.lo, p3.hi)
    g3.eval_model(p3.model_id, p3.theta, p3.n_bins, p3.n_moments)
    d3 = vup.densities_to_device(p3.dens)
    with pytest.raises(vup.VUPError) as e:
        vup.propagate_batched([grids[0], g3], [dens[0], d3], "fp32")
    assert e.value.status == vup.VUP_ERR_UNSUPPORTED
    # a grid without a model
    g0 = vup.Grid(probs[0].n, probs[0].lo, probs[0].hi)
    with pytest.raises(vup.VUPError) as e:
        vup.propagate_batched([g0], [dens[0]], "fp32")
    assert e.value.status == vup.VUP_ERR_STATE
    # densities of the wrong dimension
    with pytest.raises(vup.VUPError) as e:
        vup.propagate_batched([grids[0]], [d3], "fp32")
    assert e.value.status == vup.VUP_ERR_INVALID_ARG
    # an empty batch is a no-op
    vup.vup_propagate_batched([], [], vup.VUP_FP32, [], [])


# ------------------------------------------------- the full c5 batch
_C5 = {}


def _c5_oracle(n_sample=32):
    """The 512-instance batch the bench times, and the oracle on every row of
    a seeded sample of its instances (computed once per module)."""
    if not _C5:
        probs = I.oscillator_batch(5, n_inst=512)
        pick = np.sort(np.random.default_rng(55).choice(len(probs), size=n_sample, replace=False))
        res = {}
        for i in pick:
            p = probs[i]
            r = O.solve(p, threads=Hp.oracle_threads())
            r["scale"] = Hp.abs_moment_scale(p, r["y"], np.arange(p.K))
            res[int(i)] = r
        _C5.update(probs=probs, pick=pick, res=res)
    return _C5["probs"], _C5["pick"], _C5["res"]


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_c5_full_batch_sampled_instances(precision):
    """The real c5 batch (512 oscillator instances, sides 32..1024, K 64..8192)
    in one batched call as bench.py makes it; 32 seeded instances against the
    oracle on all of their rows, and every instance's histograms sum to 1."""
    vup = vupmod()
    probs, pick, res = _c5_oracle()
    grids, dens = [], []
    for p in probs:
        g = vup.Grid(p.n, p.lo, p.hi)
        g.eval_model(p.model_id, p.theta, p.n_bins, p.n_moments)
        grids.append(g)
        dens.append(vup.densities_to_device(p.dens))
    raws, hists = vup.propagate_batched(grids, dens, precision)
    _sync(grids)
    tol = Hp.TOL[precision]
    for i in pick:
        p, r = probs[i], res[int(i)]
        Hp.check_moments(raws[i].cpu().numpy(), r["raw"], r["scale"], tol, what=p.name)
        amb = Hp.ambiguous_points(r["y"], r["bins"], p.n_bins)
        Hp.check_hist(hists[i].cpu().numpy(), r["hist"], Hp.ambiguous_mass(p, amb, np.arange(p.K)))
    for h in hists:
        assert np.abs(h.double().sum(dim=1).cpu().numpy() - 1.0).max() <= 1e-6
    for g in grids:
        g.close()
