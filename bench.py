"""Throughput of the fused VUP hot path on GB300 (distribution-points/s).

One step = one pass of the whole hot path over the 2-D workload of the
paper's Sec. 4.1 timing experiment scaled to the configured size
(``inputs.config('c2')``: y = sin x1 + 7 sin^2 x2 on a 1024^2 midpoint grid,
K = 16384 product Gaussians, 4 moments + 256-bin histograms):
model evaluation, range, bins, counting sort, power tables, density prep,
the moment contraction, FP64 finish and the segmented histogram.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x3|fp32]
       python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import math
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1908_11246_gb300 import inputs as I  # noqa: E402

METRIC = "distribution-points/s (K*N) fused VUP"
UNIT = "dist-points/s"
WORKLOAD = ("c2: 2-D VUP, y = sin x1 + 7 sin^2 x2 on a 1024x1024 midpoint grid over [-pi,pi]^2, "
            "K=16384 product Gaussians (128x128 lattice of means), 4 raw+central moments + 256-bin histograms")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d["bf16_tflops_sustained"],
                    sm_max=d.get("sm_max_mhz", 2070.0), source="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, sm_max=2070.0, source="fallback")


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except FileNotFoundError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(prob, budget_s=12.0, threads=None):
    """The FP64 oracle as it stands, timed on the host cores on a bounded
    sample of distributions of the same workload."""
    from oracle import oracle as O
    threads = threads or (os.cpu_count() or 1)
    y = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
    b, _, _ = O.bins(y, prob.n_bins)
    rows = np.arange(threads)
    t0 = time.perf_counter()
    O.propagate(prob.n, prob.lo, prob.hi, y, b, prob.n_bins, prob.n_moments, prob.dens, rows=rows,
                threads=threads)
    t1 = time.perf_counter() - t0
    n_rows = int(max(threads, min(prob.K, threads * max(1, int(budget_s / max(t1, 1e-3))))))
    rows = np.random.default_rng(0).choice(prob.K, size=n_rows, replace=False)
    t0 = time.perf_counter()
    O.propagate(prob.n, prob.lo, prob.hi, y, b, prob.n_bins, prob.n_moments, prob.dens, rows=rows,
                threads=threads)
    dt = time.perf_counter() - t0
    return {"value": n_rows * prob.N / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n_rows} of {prob.K} distributions x all {prob.N} grid points ({dt:.1f} s)"}


def ranks_max(value, world, dist, device):
    """The largest of the ranks' values (all_reduce MAX); the value itself
    when one rank runs.  Step times are reduced this way: the job is as slow
    as its slowest replica."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds_per_step):
    """Whole-job throughput of `world` replicas that each process
    `units_per_rank` units per step (weak scaling), paced by the slowest."""
    return world * units_per_rank / seconds_per_step


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.steps is None:
        args.steps = 20
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    rows_per_step = threads
    rng = np.random.default_rng(0)
    if args.config == "c5":
        # one instance per step (drawn from the batch), `threads` of its distributions
        probs = I.oscillator_batch(5, n_inst=512)
        cache = {}

        def step():
            i = int(rng.integers(len(probs)))
            p = probs[i]
            if i not in cache:
                y = O.eval_model(p.model_id, p.theta, p.n, p.lo, p.hi)
                cache[i] = (y, O.bins(y, p.n_bins)[0])
            y, b = cache[i]
            rows = rng.choice(p.K, size=min(rows_per_step, p.K), replace=False)
            O.propagate(p.n, p.lo, p.hi, y, b, p.n_bins, p.n_moments, p.dens, rows=rows, threads=threads)
            return len(rows) * p.N
        prob = None
    else:
        prob = I.config("c2" if args.config in ("weights", "bayes") else args.config)
        if args.k or args.config == "weights":
            prob.dens = prob.dens.take(range(min(args.k or 1024, prob.K)))
        y = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
        b, _, _ = O.bins(y, prob.n_bins)

        def step():
            rows = rng.choice(prob.K, size=min(rows_per_step, prob.K), replace=False)
            O.propagate(prob.n, prob.lo, prob.hi, y, b, prob.n_bins, prob.n_moments, prob.dens, rows=rows,
                        threads=threads)
            return len(rows) * prob.N

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    units = 0
    for _ in range(args.steps):
        units += step()
    dt = time.perf_counter() - t0
    value = units / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config], "precision": "fp64 (oracle)",
                       "step": f"{rows_per_step} sampled distributions x all grid points"},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": threads,
                             "sample": f"{rows_per_step} distributions per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def traffic_for(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` recorded from an ncu
    capture (dram__bytes_read.sum + dram__bytes_write.sum) in the kernel's
    summary under profiles/, or None."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(p):
        return None
    for line in open(p):
        if line.startswith("traffic_bytes_per_launch:"):
            try:
                return float(line.split(":", 1)[1].split()[0])
            except (ValueError, IndexError):
                return None
    return None


def roofline_for(name, ms, n_work, units, pk, workload, hist_units=None):
    """Algorithmic work of one working launch of `name` divided by its event-timed duration.

    ms: device time of the group over the timed steps; n_work: the launches in
    it that do the work (the histogram's launch for the stream the device did
    not choose returns at once and is not counted); units: dist-points one
    working launch covers (every contraction launch, moments or one IPSA
    orientation, covers all K x N); hist_units: bytes one histogram pass moves
    through the SM's L1 data pipe by its algorithm (per density: 4 per point +
    4 per rest-factor row per run on the point stream; 8 of prefix sums + 4 per
    rest-factor row per interval on the interval stream; on the record stream
    4 per prefix sum a record needs -- one per bin it holds and one more, the
    intervals plus the records in all -- + 4 per rest-factor row per record)."""
    per = ms / max(n_work, 1) * 1e-3
    tr = traffic_for(name, workload)
    if name.startswith(("moments_bf16", "ipsa_bf16", "moments_tf32")):
        tf32 = name.startswith("moments_tf32")
        fl = 8.0 if name.startswith("moments_tf32_") else 24.0
        # TF32 dense = bf16 x (1.1 / 2.25), the nominal ratio of the two peaks
        ratio = 1.1 / 2.25 if tf32 else 1.0
        burst, sus = pk["bf16"] * ratio, pk["bf16_sus"] * ratio
        a = fl * units / per / 1e12
        return {"bound": "tensor", "achieved": a, "peak": burst, "unit": "TFLOP/s", "frac": a / burst,
                "peak_sustained": sus, "frac_sustained": a / sus, "traffic": tr,
                "note": f"{fl:g} tensor flops/dist-point ({'TF32' if tf32 else 'BF16x3'}, J=4) per launch; "
                        f"peak = burst {'TF32 (bf16 x 1.1/2.25)' if tf32 else 'bf16'} (the kernel runs well "
                        f"under a second), sustained beside it, of {pk['source']}"}
    if name.startswith("moments_fp32") or name.startswith("ipsa_fp32"):
        fl = 8.0  # each FP32 launch is one weighted contraction (the IPSA takes three per orientation)
        peak = pk["ffma_tflops"]
        a = fl * units / per / 1e12
        return {"bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                "traffic": tr, "note": f"{fl:g} FP32 flops/dist-point; peak = FP32 FMA throughput measured by "
                                      "vup_measure_peak(0) in this run"}
    if name.startswith("hist_seg"):
        peak = pk["gather_gbs"]
        a = (hist_units or 4.0 * units) / per / 1e9
        return {"bound": "alu", "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak, "traffic": tr,
                "note": "bytes through the L1 data pipe that the walk needs per pass (per density: point stream "
                        "4 per point + 4 per rest-factor row per run; interval stream 8 of prefix sums + 4 per "
                        "rest-factor row per interval; record stream 4 per prefix sum it needs (one per bin a "
                        "record holds + one per record) + 4 per rest-factor row "
                        "per record); peak = shared-memory 512-byte row gathers measured by "
                        "vup_measure_peak(1) in this run"}
    a = 4.0 * units / per / 1e9
    return {"bound": "hbm", "achieved": a, "peak": pk["hbm"], "unit": "GB/s", "frac": a / pk["hbm"],
            "traffic": tr, "note": f"4 B/dist-point; peak = measured copy bandwidth, of {pk['source']}"}


ROOF_GROUPS = ("moments_bf16", "moments_fp32", "moments_tf32", "ipsa_bf16", "ipsa_fp32", "hist_seg", "weights")


WORKLOADS = {
    "c2": WORKLOAD,
    "c3": ("c3: 3-D VUP, y = sin x1 + 7 sin^2 x2 + 0.1 x3^4 sin x1 on a 128^3 midpoint grid over [-pi,pi]^3, "
           "K=32768 (each axis Gaussian, uniform or truncated normal), 4 moments + 512-bin histograms"),
    "c4": ("c4: config-2 model on a 2048x2048 grid, K=65536 product Gaussians (256x256 lattice), "
           "4 moments + 256-bin histograms, then the IPSA adjoint (vector-Jacobian product w.r.t. mu, sigma)"),
    "c5": ("c5: 512 damped-oscillator instances, square grids of side log-uniform in [32,1024], "
           "K log-uniform in [64,8192], 4 moments + 128-bin histograms, one batched call per step "
           "(grids and model outputs built once)"),
    "weights": ("weights: supplied dense W (FP32 [K][N] in HBM), config-2 grid and model, K=1024, "
                "4 moments + 256-bin histograms"),
    "bayes": ("bayes: config-2 grid and model, K=16384 product Gaussians, 256 bins; the Bayes-inverted "
              "model matrix applied to the inputs: posterior mean of both axes per output bin, with H"),
    "ipsa": ("ipsa: the Sec. 5.3 IPSA example, y = x^2 + 5 sin 3x + alpha on a 1000x1000 grid over "
             "[-5,5]x[-1.5,1.5], L=1000 locations, sigma_l=0.5, sigma_alpha=0.25, 4 moments + 1000-bin "
             "histograms, then estimated values, deviation moments, the 1000-bin IPSA probability matrix "
             "and its argmax / 90% interval / marginalised fields"),
}


def packed(torch, specs, device="cuda"):
    """Tensors of the given (shape, dtype) as views of one contiguous byte
    buffer (each view 256-byte aligned); returns (buffer, views)."""
    offs, o = [], 0
    for shape, dt in specs:
        n = int(np.prod(shape)) * torch.empty((), dtype=dt).element_size()
        offs.append((o, n))
        o += -(-n // 256) * 256
    buf = torch.empty(max(o, 1), dtype=torch.uint8, device=device)
    views = [buf[a:a + n].view(dt).view(shape) for (a, n), (shape, dt) in zip(offs, specs)]
    return buf, views


class SingleGrid:
    """c2 / c3 / c4: one grid; a step evaluates the model (values, range, bins,
    sort, power tables) and propagates all K densities (plus the adjoint for c4)."""

    def __init__(self, name, k, prec, vup, torch):
        self.vup, self.torch = vup, torch
        prob = I.config("c2" if name == "bayes" else name)
        if k:
            prob.dens = prob.dens.take(range(min(k, prob.K)))
        self.prob = prob
        self.ipsa = name == "c4"
        self.sa = name == "ipsa"
        self.bayes = name == "bayes"
        self.hist_passes = 1 + prob.ndim if self.bayes else 1  # posterior means: H, then one pass per axis
        self.prec = prec
        self.g = vup.Grid(prob.n, prob.lo, prob.hi)
        K, J, B, nd_ = prob.K, prob.n_moments, prob.n_bins, prob.ndim
        f64, f32, i32 = torch.float64, torch.float32, torch.int32
        # the densities and every per-step output as views of one input and one
        # output buffer (one host copy each way end to end)
        dd = vup.densities_to_device(prob.dens)
        names = ("kind", "mu", "sigma", "lo", "hi")
        self.in_buf, views = packed(torch, [(tuple(dd[n].shape), dd[n].dtype) for n in names])
        self.dev = dict(zip(names, views))
        for n in names:
            self.dev[n].copy_(dd[n])
        del dd
        self.ds = vup.make_densities(self.dev)
        self.nd = 1000
        specs = {"hist": ((K, B), f32)} if self.bayes else \
            {"raw": ((K, J), f64), "cen": ((K, J), f64), "hist": ((K, B), f32)}
        if self.ipsa:
            specs.update(dmu=((K, 2), f32), dsg=((K, 2), f32))
        if self.bayes:
            specs.update(post=((K, B, nd_), f32))
        if self.sa:
            specs.update(yref=((K,), f64), dev_m=((K, J), f64), mat=((K, self.nd), f32), am=((K,), i32),
                         ci=((K, 2), i32), glob=((self.nd,), f64))
        self.out_buf, outs = packed(torch, list(specs.values()))
        for name, v in zip(specs, outs):
            setattr(self, name, v)
        if self.ipsa:
            self.grad = torch.ones((K, J), dtype=f64, device="cuda")
        if self.sa:
            self.g.eval_model(prob.model_id, prob.theta, B, J)
            info = self.g.info()
            self.span = info.ymax - info.ymin
            self.centres = self.dev["mu"].contiguous()
        self.units = K * prob.N
        self.K = K

    def step(self, stream):
        v, p = self.vup, self.prob
        v.vup_eval_model(self.g.h, p.model_id, p.theta, p.n_bins, p.n_moments, stream)
        if self.bayes:
            v.vup_posterior_means(self.g.h, self.ds, self.hist, self.post, stream)
            return
        if self.ipsa:
            # forward pass and sensitivities in one call (one density preparation)
            v.vup_propagate_ipsa(self.g.h, self.ds, self.prec, self.raw, self.cen, self.hist, self.dmu, self.dsg,
                                 self.grad, stream)
        else:
            v.vup_propagate(self.g.h, self.ds, self.prec, self.raw, self.cen, self.hist, stream)
        if self.sa:
            v.vup_model_at(self.g.h, self.centres, self.yref, stream)
            v.vup_deviation_moments(self.g.h, self.raw, self.yref, self.dev_m, stream)
            v.vup_ipsa_matrix(self.g.h, self.hist, self.yref, self.nd, -self.span, self.span, self.mat, stream)
            v.vup_sa_fields(self.mat, 0.9, None, self.am, self.ci, self.glob, stream)

    def sync(self):
        self.g.sync()

    def hist_grids(self):
        return [(self.g, self.K)]

    def e2e(self):
        """Host buffers: the densities copied in and every output of the step
        copied back, each step (one copy each way: the packed buffers)."""
        torch = self.torch
        in_h = self.in_buf.cpu().pin_memory()
        out_h = torch.empty_like(self.out_buf, device="cpu").pin_memory()
        bi, bo = in_h.numel(), out_h.numel()

        def run(stream):
            self.in_buf.copy_(in_h, non_blocking=True)
            self.step(stream)
            out_h.copy_(self.out_buf, non_blocking=True)
        return run, bi, bo


class Batched:
    """c5: many uneven instances, one batched call (graph replay) per step."""

    def __init__(self, prec, vup, torch):
        self.vup, self.torch = vup, torch
        self.probs = I.oscillator_batch(5, n_inst=512)
        self.grids = []
        for p in self.probs:
            g = vup.Grid(p.n, p.lo, p.hi)
            g.eval_model(p.model_id, p.theta, p.n_bins, p.n_moments)
            self.grids.append(g)
        # every instance's densities and outputs are views of a few contiguous
        # device buffers (each view 256-byte aligned), so that a host round trip
        # moves them with one copy per buffer
        nd = 2
        pad = lambda n, a: -(-n // a) * a
        din = [pad(p.K * nd, 32) for p in self.probs]
        dr = [pad(p.K * p.n_moments, 32) for p in self.probs]
        dh = [pad(p.K * p.n_bins, 64) for p in self.probs]
        self.kind_buf = torch.zeros(sum(din), dtype=torch.uint8, device="cuda")
        self.par_buf = torch.zeros((4, sum(din)), dtype=torch.float64, device="cuda")
        self.raw_buf = torch.empty(sum(dr), dtype=torch.float64, device="cuda")
        self.hist_buf = torch.empty(sum(dh), dtype=torch.float32, device="cuda")
        self.dev, raws, hists = [], [], []
        oi = orr = oh = 0
        for p, a, b, c in zip(self.probs, din, dr, dh):
            n = p.K * nd
            d = dict(kind=self.kind_buf[oi:oi + n].view(p.K, nd))
            for r, name in enumerate(("mu", "sigma", "lo", "hi")):
                d[name] = self.par_buf[r, oi:oi + n].view(p.K, nd)
            for name, v in vup.densities_to_device(p.dens).items():
                d[name].copy_(v)
            self.dev.append(d)
            raws.append(self.raw_buf[orr:orr + p.K * p.n_moments].view(p.K, p.n_moments))
            hists.append(self.hist_buf[oh:oh + p.K * p.n_bins].view(p.K, p.n_bins))
            oi, orr, oh = oi + a, orr + b, oh + c
        self.prec = prec
        self.out = (raws, hists)
        self.units = sum(p.K * p.N for p in self.probs)
        self.K = sum(p.K for p in self.probs)
        self.call = vup.BatchedArgs([g.h for g in self.grids], [vup.make_densities(d) for d in self.dev],
                                    self.out[0], self.out[1])

    def step(self, stream):
        self.call(self.prec, stream)

    def hist_grids(self):
        return [(g, p.K) for g, p in zip(self.grids, self.probs)]

    def sync(self):
        for g in self.grids:
            g.sync()

    def e2e(self):
        """Host buffers: every instance's densities copied in and every output
        copied back, each step (one copy per contiguous buffer)."""
        torch = self.torch
        ins = [self.kind_buf, self.par_buf]
        outs = [self.raw_buf, self.hist_buf]
        ins_h = [x.cpu().pin_memory() for x in ins]
        outs_h = [torch.empty_like(x, device="cpu").pin_memory() for x in outs]
        bi = sum(x.numel() * x.element_size() for x in ins_h)
        bo = sum(x.numel() * x.element_size() for x in outs_h)

        def run(stream):
            for d, h in zip(ins, ins_h):
                d.copy_(h, non_blocking=True)
            self.step(stream)
            for h, d in zip(outs_h, outs):
                h.copy_(d, non_blocking=True)
        return run, bi, bo


class Weights:
    """Supplied-W path: dense W [K][N] FP32 resident in HBM, moments + histograms."""

    def __init__(self, k, vup, torch):
        self.vup, self.torch = vup, torch
        prob = I.config("c2")
        prob.dens = prob.dens.take(range(k or 1024))
        self.prob = prob
        self.g = vup.Grid(prob.n, prob.lo, prob.hi)
        self.g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
        K, (n0, n1) = prob.K, prob.n
        # input generation (not the measured path): normalised product Gaussians
        x0 = torch.linspace(prob.lo[0], prob.hi[0], n0 + 1, dtype=torch.float64, device="cuda")
        x1 = torch.linspace(prob.lo[1], prob.hi[1], n1 + 1, dtype=torch.float64, device="cuda")
        x0, x1 = 0.5 * (x0[1:] + x0[:-1]), 0.5 * (x1[1:] + x1[:-1])
        mu = torch.as_tensor(prob.dens.mu, device="cuda")
        sg = torch.as_tensor(prob.dens.sigma, device="cuda")
        w0 = torch.exp(-0.5 * ((x0[None, :] - mu[:, :1]) / sg[:, :1]) ** 2)
        w1 = torch.exp(-0.5 * ((x1[None, :] - mu[:, 1:]) / sg[:, 1:]) ** 2)
        w0 = w0 / w0.sum(1, keepdim=True)
        w1 = w1 / w1.sum(1, keepdim=True)
        self.W = torch.empty((K, n0 * n1), dtype=torch.float32, device="cuda")
        for k0 in range(0, K, 64):
            blk = (w0[k0:k0 + 64, :, None] * w1[k0:k0 + 64, None, :]).reshape(-1, n0 * n1)
            self.W[k0:k0 + 64] = blk.float()
        del w0, w1
        self.raw = torch.empty((K, prob.n_moments), dtype=torch.float64, device="cuda")
        self.hist = torch.empty((K, prob.n_bins), dtype=torch.float32, device="cuda")
        self.units = K * prob.N
        self.K = K

    def hist_grids(self):
        return []

    def step(self, stream):
        self.vup.vup_propagate_weights(self.g.h, self.W, self.raw, self.hist, stream)

    def sync(self):
        self.g.sync()

    def e2e(self):
        torch = self.torch
        Wh = self.W.cpu().pin_memory()
        outs = [self.raw, self.hist]
        outs_h = [torch.empty_like(x, device="cpu").pin_memory() for x in outs]
        bi = Wh.numel() * Wh.element_size()
        bo = sum(x.numel() * x.element_size() for x in outs_h)

        def run(stream):
            self.W.copy_(Wh, non_blocking=True)
            self.step(stream)
            for h, d in zip(outs_h, outs):
                h.copy_(d, non_blocking=True)
        return run, bi, bo


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: enough for a timed region of about 1.5 s, 20 to 2000)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp32", "tf32x3", "tf32"])
    ap.add_argument("--config", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--k", type=int, default=0, help="use the first K densities of the workload (0: all)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32-arm", action="store_true", help="skip the plain FP32 comparator run")
    ap.add_argument("--hist-stream", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="histogram stream: -1 automatic, 0 sorted points, 1 sorted intervals, 2 records")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    from paper_1908_11246_gb300 import build as B
    B.build()
    from paper_1908_11246_gb300 import vup

    pk = peaks()
    # measured ceilings of the CUDA-core resources (FP32 FMA, shared-memory gathers)
    pk["ffma_tflops"] = vup.vup_measure_peak(0) / 1e12
    pk["gather_gbs"] = vup.vup_measure_peak(1) / 1e9
    prec = vup.PRECISIONS[args.precision]
    if args.config == "c5":
        work = Batched(prec, vup, torch)
    elif args.config == "weights":
        work = Weights(args.k, vup, torch)
    else:
        work = SingleGrid(args.config, args.k, prec, vup, torch)
    stream = torch.cuda.current_stream()
    if args.hist_stream != -1:
        for g, _ in work.hist_grids():
            g.set_hist_stream(args.hist_stream)

    for _ in range(max(3, args.warmup)):
        work.step(stream)
    work.sync()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    if args.steps is None:
        # default step count: a timed region long enough for several clock
        # samples (one more untimed step sizes it)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        work.step(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        est = ranks_max(max(e0.elapsed_time(e1), 1e-3), world, dist, "cuda")
        args.steps = int(min(2000, max(20, math.ceil(1500.0 / est))))

    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # the batched path replays one CUDA graph per step; its per-stage times
    # come from a separate pass below (profiling makes it launch stage by stage)
    profile_live = args.config != "c5"
    if profile_live:
        vup.vup_profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        work.step(stream)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    if not profile_live:
        vup.vup_profile(True)
        for s in range(args.steps):
            flush.zero_()
            work.step(stream)
        torch.cuda.synchronize()
    vup.vup_profile(False)
    prof = vup.vup_profile_read()
    work.sync()
    t_ms = ranks_max(sum(a.elapsed_time(b) for a, b in ev), world, dist, "cuda")
    ms_step = t_ms / args.steps
    value = job_rate(work.units, world, ms_step * 1e-3)

    # end-to-end through the public API with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        run, bi, bo = work.e2e()
        n_e2e = max(3, args.steps // 2)
        run(stream)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(n_e2e):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run(stream)
            torch.cuda.synchronize()
            tot += time.perf_counter() - t0
        work.sync()
        tot = ranks_max(tot, world, dist, "cuda")
        e2e = {"value": job_rate(work.units, world, tot / n_e2e), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": 1e3 * tot / n_e2e}

    # the plain FP32 GPU path on the same workload (the metric's comparator):
    # a shorter timed run after the main one, its contraction timed alone
    fp32_arm = None
    if args.precision != "fp32" and not args.no_fp32_arm and args.config not in ("weights", "bayes"):
        work.prec = vup.PRECISIONS["fp32"]
        n32 = max(3, args.steps // 4)
        for _ in range(3):
            work.step(stream)
        work.sync()
        torch.cuda.synchronize()
        if profile_live:
            vup.vup_profile(True)
        e32 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n32)]
        for s in range(n32):
            flush.zero_()
            e32[s][0].record(stream)
            work.step(stream)
            e32[s][1].record(stream)
        torch.cuda.synchronize()
        if not profile_live:  # the batched graph launches stage by stage while profiled
            vup.vup_profile(True)
            for s in range(n32):
                flush.zero_()
                work.step(stream)
            torch.cuda.synchronize()
        vup.vup_profile(False)
        prof32 = vup.vup_profile_read()
        work.sync()
        work.prec = prec
        ms32 = ranks_max(sum(a.elapsed_time(b) for a, b in e32) / n32, world, dist, "cuda")
        v32 = job_rate(work.units, world, ms32 * 1e-3)

        def contraction_ms(pr, n):
            # the contraction launches: moments and (c4) sensitivities, tensor-core or SIMT,
            # single or batched; not the FP64 finishes
            return sum(v[1] for k, v in pr.items() if k.startswith(("moments_", "ipsa_")) and
                       ("_tc" in k or "_simt" in k)) / n
        c_main, c_32 = contraction_ms(prof, args.steps), contraction_ms(prof32, n32)
        fp32_arm = {"value": v32, "unit": UNIT, "ms_per_step": ms32, "steps": n32,
                    "factor_step": value / v32, "contraction_ms": {args.precision: c_main, "fp32": c_32},
                    "factor_contraction": (c_32 / c_main) if c_main > 0 else None,
                    "note": "the same workload with the plain FP32 CUDA-core contraction (8-term FP32 chains, "
                            "compensated folds), timed the same way after the main run; contraction_ms "
                            "sums the contraction launches per step (profiled pass for c5)"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    per_step = {k: {"launches": v[0] / args.steps, "ms_per_step": v[1] / args.steps} for k, v in prof.items()}
    wl = args.config + (f"_k{work.K}" if args.k else "")
    # dominant: the costliest group with a roofline (groups on the second stream
    # overlap others and are not candidates)
    cands = {k: v for k, v in prof.items() if k.startswith(ROOF_GROUPS)}
    dominant = max(cands.items(), key=lambda kv: kv[1][1])[0] if cands else None
    # gathers of one histogram launch on the stream each grid's layout chose
    hist_units, streams = 0, set()
    points_only = getattr(work, "bayes", False)  # posterior means walk the point stream
    for g, K in work.hist_grids():
        info = g.info()
        if info.ndim >= 2:
            mode = 0 if points_only else info.hist_stream
            streams.add(("points", "intervals", "records")[mode])
            nf = info.ndim - 1  # rest-factor rows per run, interval or record
            if mode == 2:
                hist_units += K * (4 * (info.hist_intervals + info.hist_records) + 4 * nf * info.hist_records)
            elif mode == 1:
                hist_units += K * info.hist_intervals * (8 + 4 * nf)
            else:
                hist_units += K * (4 * info.N + 4 * nf * info.hist_runs)
    def n_work(k, launches):
        # histogram: one working launch per pass (the other stream's launch exits at once)
        if k.startswith("hist_seg"):
            return args.steps * getattr(work, "hist_passes", 1)
        # the supplied-weights group is one pass per step over several launches
        # (power table, the W stream, the finish): its bytes are per pass
        if k.startswith("weights"):
            return args.steps
        return launches

    def roof_of(k, v):
        return roofline_for(k, v[1], n_work(k, v[0]), work.units, pk, wl, hist_units)
    roof = roof_of(dominant, prof[dominant]) if dominant else None
    if roof:
        roof["kernel"] = dominant
    kern_roof = {k: roof_of(k, v) for k, v in prof.items() if k.startswith(ROOF_GROUPS)}
    stage = {"model_eval_bins_sort_tables": 0.0, "moments": 0.0, "histogram": 0.0, "ipsa": 0.0, "other": 0.0}
    for k, v in per_step.items():
        if k.startswith(("model_eval", "range_bins", "layout_sort", "power_table")):
            stage["model_eval_bins_sort_tables"] += v["ms_per_step"]
        elif k.startswith(("moments", "density_prep")):
            stage["moments"] += v["ms_per_step"]
        elif k.startswith("hist"):
            stage["histogram"] += v["ms_per_step"]
        elif k.startswith("ipsa"):
            stage["ipsa"] += v["ms_per_step"]
        else:
            stage["other"] += v["ms_per_step"]
    # the supplied-weights path computes in FP32 (FP64 finish) whatever --precision says
    precision = "fp32" if args.config == "weights" else args.precision
    cfg = {"workload": WORKLOADS[args.config], "dist_points_per_step": work.units, "K": work.K,
           "precision": precision, "parallelism": f"replicas x{world} (no collective)",
           "l2": "flushed before every timed step (256 MB write, outside the step events)"}
    if args.k:
        cfg["k_subset"] = work.K
    if streams:
        cfg["hist_stream"] = "+".join(sorted(streams))
    if hasattr(work, "prob"):
        cfg.update({"N": work.prob.N, "bins": work.prob.n_bins, "moments": work.prob.n_moments})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"bf16x3": "bf16", "tf32x3": "tf32", "tf32": "tf32"}.get(precision, "f32"),
        "data": "synthetic",
        "config": cfg,
        "roofline": roof,
        "kernels": {"per_step": per_step, "stage_ms_per_step": stage, "roofline": kern_roof,
                    "timing": ("CUDA events per kernel group inside the timed region, on each group's own "
                               "stream: the layout build runs on a second stream beside the density "
                               "preparation and the contraction, the prefix tiles and the FP64 moments finish "
                               "on a third (the finish waits there for SM room beside the histogram), so "
                               "group spans overlap and can add up to more than ms_per_step") if profile_live
                    else "per-stage CUDA events from a second pass of the same steps (stage by stage)"},
        "fp32_arm": fp32_arm,
        "measured_ceilings": {"fp32_ffma_tflops": pk["ffma_tflops"], "smem_gather_gbs": pk["gather_gbs"],
                              "how": "vup_measure_peak: FMA chains and 512-byte shared-memory row gathers on "
                                     "every SM, CUDA events, in this run"},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "clocks": clk,
        "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline and hasattr(work, "prob") and args.config != "weights":
        line["cpu_baseline"] = cpu_baseline(work.prob)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
