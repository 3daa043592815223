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


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prob = I.config(args.config)
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    y = O.eval_model(prob.model_id, prob.theta, prob.n, prob.lo, prob.hi)
    b, _, _ = O.bins(y, prob.n_bins)
    rows_per_step = threads
    rng = np.random.default_rng(0)

    def step():
        rows = rng.choice(prob.K, size=rows_per_step, replace=False)
        O.propagate(prob.n, prob.lo, prob.hi, y, b, prob.n_bins, prob.n_moments, prob.dens, rows=rows,
                    threads=threads)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = args.steps * rows_per_step * prob.N / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "K": prob.K, "N": prob.N, "bins": prob.n_bins,
                       "step": f"{rows_per_step} sampled distributions x all grid points"},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": threads,
                             "sample": f"{rows_per_step} distributions per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def roofline_for(name, ms, launches, prob, pk, clk_mhz):
    """Algorithmic work of one launch of `name` divided by its event-timed duration."""
    KN = prob.K * prob.N
    per = ms / max(launches, 1) * 1e-3
    sms = 152
    if name.startswith("moments_bf16"):
        a = 24.0 * KN / per / 1e12   # 3 BF16 products x 2J flops per dist-point
        return {"bound": "tensor", "achieved": a, "peak": pk["bf16_sus"], "unit": "TFLOP/s",
                "frac": a / pk["bf16_sus"], "traffic": None,
                "note": f"24 tensor flops/dist-point (BF16x3, J=4), peak = sustained bf16 ({pk['source']})"}
    if name.startswith("moments_fp32"):
        peak = sms * 128 * 2 * clk_mhz * 1e6 / 1e12
        a = 8.0 * KN / per / 1e12
        return {"bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                "traffic": None, "note": "8 FP32 flops/dist-point; peak = 152 SM x 128 FMA x 2 x median SM clock"}
    if name.startswith("hist"):
        peak = sms * 128 * clk_mhz * 1e6 / 1e9
        a = 4.0 * KN / per / 1e9
        return {"bound": "alu", "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak, "traffic": None,
                "note": "one 4-byte shared-memory factor gather per dist-point; peak = 152 SM x 128 B/clk "
                        "shared-memory bandwidth x median SM clock"}
    a = 4.0 * KN / per / 1e9
    return {"bound": "hbm", "achieved": a, "peak": pk["hbm"], "unit": "GB/s", "frac": a / pk["hbm"],
            "traffic": None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp32"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
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

    prob = I.config(args.config)
    pk = peaks()
    prec = vup.PRECISIONS[args.precision]
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    dev = vup.densities_to_device(prob.dens)
    dstruct = vup.make_densities(dev)
    K, J, Bn = prob.K, prob.n_moments, prob.n_bins
    raw = torch.empty((K, J), dtype=torch.float64, device="cuda")
    cen = torch.empty((K, J), dtype=torch.float64, device="cuda")
    hist = torch.empty((K, Bn), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        vup.vup_eval_model(g.h, prob.model_id, prob.theta, Bn, J, stream)
        vup.vup_propagate(g.h, dstruct, prec, raw, cen, hist, stream)

    for _ in range(max(3, args.warmup)):
        step()
    g.sync()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    vup.vup_profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        step()
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    vup.vup_profile(False)
    clk = clocks.stop()
    prof = vup.vup_profile_read()
    g.sync()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    t = torch.tensor([t_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_ms = float(t.item())
    ms_step = t_ms / args.steps
    value = world * K * prob.N / (ms_step * 1e-3)

    # end-to-end through the public API with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        host = {k: v.cpu().pin_memory() for k, v in dev.items()}
        raw_h = torch.empty_like(raw, device="cpu").pin_memory()
        cen_h = torch.empty_like(cen, device="cpu").pin_memory()
        hist_h = torch.empty_like(hist, device="cpu").pin_memory()
        bi = sum(v.numel() * v.element_size() for v in host.values())
        bo = sum(x.numel() * x.element_size() for x in (raw_h, cen_h, hist_h))
        n_e2e = max(3, args.steps // 2)

        def e2e_step():
            for k, v in host.items():
                dev[k].copy_(v, non_blocking=True)
            step()
            raw_h.copy_(raw, non_blocking=True)
            cen_h.copy_(cen, non_blocking=True)
            hist_h.copy_(hist, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(n_e2e):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            tot += time.perf_counter() - t0
        e2e = {"value": world * K * prob.N / (tot / n_e2e), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": 1e3 * tot / n_e2e}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    clk_mhz = clk["sm_mhz"] if clk else pk["sm_max"]
    per_step = {k: {"launches": v[0] / args.steps, "ms_per_step": v[1] / args.steps} for k, v in prof.items()}
    dominant = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    roof = roofline_for(dominant, prof[dominant][1], prof[dominant][0], prob, pk, clk_mhz) if dominant else None
    if roof:
        roof["kernel"] = dominant
    kern_roof = {k: roofline_for(k, v[1], v[0], prob, pk, clk_mhz)
                 for k, v in prof.items() if k.startswith(("moments_bf16", "moments_fp32", "hist_seg"))}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if args.precision == "bf16x3" else "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "K": K, "N": prob.N, "bins": Bn, "moments": J,
                   "precision": args.precision, "parallelism": f"replicas x{world} (K-sharded, no collective)",
                   "l2": "flushed before every timed step (256 MB write, outside the step events)"},
        "roofline": roof,
        "kernels": {"per_step": per_step, "roofline": kern_roof},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "clocks": clk,
        "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
