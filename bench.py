#!/usr/bin/env python
"""Benchmark: gap-certified Lasso solves/s of the GAP SAFE coordinate-descent
path on one GB300 (or N independent replicas, one per GPU).

Workload (one step): the Toeplitz-correlated design 500 x 50000 (corr 0.5^|i-j|,
unit-norm columns, FP32 storage), beta* 50-sparse N(0,1), SNR 5, a 100-point
geometric grid from lambda_max to lambda_max/1000, a GAP SAFE check every 10
passes, stop at gap <= 1e-6 ||y||^2 -- one full path = 100 (problem, lambda)
solves, each certified by its duality gap.  Inputs are seeded synthetic data
resident in HBM; L2 is flushed (a 512 MiB write) before every timed step.

Keys beyond the base contract:
  roofline      the path kernel's algorithmic bytes (x_columns * n * 4 per
                launch, from the solver's own counters) / its event-timed
                duration, against the measured HBM copy peak
  cpu_baseline  the FP64 oracle on the host cores, a bounded sample of the
                same path (its first 50 lambdas)
  xtr_pass      the standalone correlation pass c = X^T r (the check's HBM
                stream) timed per launch, L2 flushed, against the HBM peak
  tuned_vs_plain  the batched solver (256 stability-selection problems x 50
                lambdas) against the plain single-problem path on a sample
  e2e           the same metric through the C-ABI with the inputs copied from
                pinned host memory and beta/stats copied back inside the step
  clocks        nvidia-smi SM clocks and throttle reasons sampled during the
                timed region
``--impl reference`` times the oracle alone (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gap-certified Lasso solves/s at gap<=1e-6"
CPU_SAMPLE_T = 50


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lambdas", type=int, default=0,
                    help="solve only the first K lambdas of the grid (a smaller case for profiling)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the correlation-pass roofline and the tuned-vs-plain comparison")
    ap.add_argument("--no-tuned", action="store_true", help="skip the tuned-vs-plain comparison")
    ap.add_argument("--learned", type=int, default=32768, metavar="N_TRAIN",
                    help="learned warm start on the 300 x 10000 design: train on N_TRAIN solver solutions "
                         "(0 skips it), then solve --learned-eval held-out responses from zero and from the net")
    ap.add_argument("--learned-eval", type=int, default=1024, metavar="N_EVAL")
    ap.add_argument("--learned-epochs", type=int, default=10)
    ap.add_argument("--large-sample", type=int, default=16, metavar="B",
                    help="right-hand sides of the 2000 x 100000 multi-RHS workload solved by the tuned batched "
                         "solver for the large tuned-vs-plain line (0 skips it)")
    ap.add_argument("--plain-sample", type=int, default=8,
                    help="problems of the batched workload timed one at a time on the plain path")
    ap.add_argument("--screen-rule", type=int, choices=[0, 1], default=0,
                    help="0: GAP SAFE sphere (default); 1: sphere and GAP SAFE dome")
    ap.add_argument("--enet-alpha", type=float, default=1.0,
                    help="Elastic-Net mixing a in (0, 1]; 1 (default) is the Lasso")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_ranks(total_ms, solves, device=None):
    """Whole-job figures over the ranks of an initialised process group: the
    timed region is the slowest rank's (max), the certified solves add up.
    Without a group (one process) the inputs come back unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), int(solves)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([float(solves)], dtype=torch.float64, device=device)
    dist.all_reduce(s)
    return float(t.item()), int(round(float(s.item())))


def _workload(screen_rule=0, enet_alpha=1.0):
    import gen
    return dict(gen.workload2(), screen_rule=screen_rule, enet_alpha=enet_alpha)


def _config(w):
    return {"workload": f"{w['name']}: Toeplitz corr 0.5^|i-j| design {w['n']}x{w['p']} FP32 unit-norm, "
                        f"beta* 50-sparse N(0,1), SNR 5, T={w['T']} geometric grid lambda_max..lambda_max/1000, "
                        f"check every {w['f']} passes, gap<=1e-6*||y||^2",
            "n": w["n"], "p": w["p"], "T": w["T"], "screen_period": w["f"], "gap_tol_rel": w["tol"],
            "screen_rule": "dome" if w.get("screen_rule", 0) == 1 else "sphere",
            "enet_alpha": w.get("enet_alpha", 1.0),
            "l2": "flushed (512 MiB write) before every timed step",
            "parallelism": "replicas (one independent path per GPU)"}


def _oracle_sample(w, T=CPU_SAMPLE_T):
    """FP64 oracle on the first T lambdas of the same path; returns (solves, s)."""
    import oracle
    oracle.build()
    ratios = oracle.lambda_ratios(w["T"], w["delta"])[:T]
    t0 = time.perf_counter()
    out = oracle.lasso_path(w["XT"], w["y"], ratios, n=w["n"], screen_period=w["f"], gap_tol_rel=w["tol"],
                            screen_rule=w.get("screen_rule", 0), enet_alpha=w.get("enet_alpha", 1.0))
    dt = time.perf_counter() - t0
    return int((out["stats"]["converged"] == 1).sum()), dt


ENET_ORACLE_NOTE = ("the oracle's Elastic-Net builds the (n+p) x p augmented design at every lambda: "
                    "20 GB at 500 x 50000, so it is not timed at this size")


def _cpu_baseline(w):
    if w.get("enet_alpha", 1.0) < 1.0:
        return {"unavailable": ENET_ORACLE_NOTE}
    solves, dt = _oracle_sample(w)
    return {"value": solves / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle (plain C, single thread) on the first {CPU_SAMPLE_T} of the {w['T']} lambdas "
                      f"of the same path ({solves} certified solves in {dt:.2f} s); the later lambdas need more "
                      f"passes, so this sample favours the oracle"}


class _Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        sm = [s for s, _, _ in rows]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(m for _, m, _ in rows), "reasons": reasons,
                "samples": len(rows)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def _traffic_record():
    """DRAM bytes per launch of the path kernel from the committed ncu summary,
    valid only while the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "path_kernel_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    return rec if rec.get("source_sha256") == path_kernel_sha() else None


def path_kernel_sha():
    """sha256 over the sources the path kernel is compiled from."""
    h = hashlib.sha256()
    for f in ("path_kernel.cuh", "gram_chain.cuh", "cd_common.cuh", "dfloat.cuh", "device_util.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1505_03410_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    w = _workload(args.screen_rule, args.enet_alpha)
    if args.enet_alpha < 1.0:
        print(json.dumps({"impl": "reference", "unavailable": ENET_ORACLE_NOTE}), flush=True)
        return
    for _ in range(args.warmup):
        _oracle_sample(w)
    total_s, total_solves, times = 0.0, 0, []
    for _ in range(args.steps):
        solves, dt = _oracle_sample(w)
        total_s += dt
        total_solves += solves
        times.append(dt)
    v = total_solves / total_s
    sample = (f"FP64 oracle (plain C, single thread) on the first {CPU_SAMPLE_T} of the {w['T']} lambdas of "
              f"the same path per step")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)", "config": _config(w),
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1505_03410_gb300.build import build
    build()
    import paper_1505_03410_gb300 as pkg

    w = _workload(args.screen_rule, args.enet_alpha)
    n, p, T = w["n"], w["p"], w["T"]
    ratios_h = pkg.lasso_lambda_grid(T, w["delta"])
    if 0 < args.lambdas < T:
        T = args.lambdas
        ratios_h = ratios_h[:T].copy()
        w = dict(w, T=T, name=w["name"] + f"-first{T}")
    XT = torch.from_numpy(w["XT"]).to(dev)
    y = torch.from_numpy(w["y"]).to(dev)
    ratios = torch.from_numpy(ratios_h).to(dev)
    opts = pkg.lasso_default_opts(screen_period=w["f"], gap_tol_rel=w["tol"], screen_rule=args.screen_rule,
                                  enet_alpha=args.enet_alpha)
    words = (p + 31) // 32
    beta_out = torch.empty((T, p), dtype=torch.float64, device=dev)
    mask_out = torch.empty((T, words), dtype=torch.int32, device=dev)
    stats = torch.empty(T * pkg.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    wsb = pkg.lasso_path_workspace_size(n, p, pkg.LASSO_F32, opts)
    work = torch.empty(wsb, dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(Xp, yp, rp):
        pkg.lasso_path(Xp, pkg.LASSO_F32, n, p, w["ldx"], yp, rp, T, None, opts, beta_out.data_ptr(),
                       mask_out.data_ptr(), stats.data_ptr(), work.data_ptr(), wsb, stream.cuda_stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        step(XT.data_ptr(), y.data_ptr(), ratios.data_ptr())
    torch.cuda.synchronize()

    clocks = _Clocks(dev.index)
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(stream)
    solves = 0
    xcols = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        step(XT.data_ptr(), y.data_ptr(), ratios.data_ptr())
        ev[k][1].record(stream)
    t_all1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    phases = pkg.lasso_path_phase_cycles(work.data_ptr(), stream.cuda_stream)
    st = pkg.stats_to_numpy(stats)
    solves_per_step = int((st["status"] == 0).sum())
    solves = solves_per_step * args.steps
    xcols = int(st["x_columns"].sum())
    total_ms = t_all0.elapsed_time(t_all1)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms, solves_all = aggregate_ranks(total_ms, solves, dev)
    value = solves_all / (total_ms / 1e3)

    # e2e: inputs from pinned host memory, results back to the host, inside the step
    XT_h = torch.from_numpy(w["XT"]).pin_memory()
    y_h = torch.from_numpy(w["y"]).pin_memory()
    r_h = torch.from_numpy(ratios_h).pin_memory()
    beta_h = torch.empty((T, p), dtype=torch.float64).pin_memory()
    stats_h = torch.empty(stats.numel(), dtype=torch.uint8).pin_memory()
    Xd = torch.empty_like(XT)
    yd = torch.empty_like(y)
    rd = torch.empty_like(ratios)
    e2e_steps = max(1, args.steps)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_solves = 0
    for _ in range(e2e_steps):
        Xd.copy_(XT_h, non_blocking=True)
        yd.copy_(y_h, non_blocking=True)
        rd.copy_(r_h, non_blocking=True)
        step(Xd.data_ptr(), yd.data_ptr(), rd.data_ptr())
        beta_h.copy_(beta_out, non_blocking=True)
        stats_h.copy_(stats, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        e2e_solves += int((stats_h.numpy().view(pkg.STATS_DTYPE)["status"] == 0).sum())
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    h2d = XT_h.numel() * XT_h.element_size() + y_h.numel() * 8 + r_h.numel() * 8
    d2h = beta_h.numel() * 8 + stats_h.numel()
    e2e_ms, e2e_solves = aggregate_ranks(e2e_ms, e2e_solves, dev)
    e2e_value = e2e_solves / (e2e_ms / 1e3)

    peaks = _peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    bytes_per_launch = xcols * n * 4.0
    achieved = bytes_per_launch / (statistics.mean(launch_ms) / 1e3) / 1e9
    tr = _traffic_record()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "kernel": "path_kernel (one cooperative launch per path)",
                "bytes_per_launch": bytes_per_launch, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "note": "the path is bound by the latency of the sequential coordinate chain on one SM, "
                        "not by HBM; this is the fraction of the copy peak the algorithmic bytes reach"}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32x2+f64",
            "data": "synthetic (seeded), inputs resident in HBM", "config": _config(w),
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "steps": e2e_steps},
            "gpu_launches": 5 * args.steps, "clocks": clk,
            "phase_split": _phase_split(phases),
            "solves_per_step": solves_per_step, "epochs_per_step": int(st["epochs"].sum()),
            "checks_per_step": int(st["checks"].sum())}
    if ws == 1 and not args.no_extras:
        line["xtr_pass"] = [
            _xtr_pass(pkg, torch, dev, stream, flush, peak, peak_src, XT, n, p, w["ldx"],
                      "toeplitz-500x50000-f32 (100 MB, the bench design)")]
        g = torch.Generator(device=dev)
        g.manual_seed(1005)
        Xbig = torch.randn((100000, 2000), generator=g, device=dev, dtype=torch.float32)
        line["xtr_pass"].append(_xtr_pass(pkg, torch, dev, stream, flush, peak, peak_src, Xbig, 2000, 100000, 2000,
                                          "gaussian-2000x100000-f32 (800 MB, the large multi-RHS design)"))
        del Xbig
        line["tc_gemm"] = _tc_gemm(pkg, torch, dev, stream, flush, peaks)
        if not args.no_tuned:
            line["tuned_vs_plain"] = _tuned_vs_plain(pkg, torch, dev, stream, flush, args.plain_sample)
    if ws == 1 and args.learned > 0 and not args.no_extras:
        line["learned_warm_start"] = _learned(pkg, torch, dev, stream, args.learned, epochs=args.learned_epochs,
                                              n_eval=args.learned_eval)
    if ws == 1 and args.large_sample > 0 and not args.no_extras and not args.no_tuned:
        line["tuned_vs_plain_large"] = _tuned_vs_plain_large(pkg, torch, dev, stream, flush, args.large_sample)
    if ws == 1 and not args.no_extras:
        line["bound_audit"] = _audit(pkg, torch, dev, w, XT, y, ratios, T)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(w)
        if "value" in line["cpu_baseline"] and T >= CPU_SAMPLE_T:
            line["cpu_baseline"]["gpu_same_sample"] = _gpu_sample(pkg, torch, dev, stream, flush, w, XT, y,
                                                                  ratios_h[:CPU_SAMPLE_T], opts)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _phase_split(ph):
    """Share of the path kernel's time per phase (cycles of CTA 0's first
    thread, accumulated over the last launch's whole path)."""
    keys = ("check", "chain", "verify", "round_end", "pass_end", "other")
    tot = float(sum(ph[k] for k in keys)) or 1.0
    out = {k: round(ph[k] / tot, 4) for k in keys}
    out["chain_entries"] = ph["chain_entries"]
    out["rollbacks"] = ph["rollbacks"]
    out["cycles"] = int(tot)
    return out


def _audit(pkg, torch, dev, w, XT, y, ratios, T):
    """One untimed run of the same path with audit_bounds = 1: the largest
    |c~_j - x_j^T rho| / E_j of the FP32 correlations over every check of every
    lambda (row a11: <= 1 when every forward-error bound holds)."""
    opts = pkg.lasso_default_opts(screen_period=w["f"], gap_tol_rel=w["tol"], screen_rule=w.get("screen_rule", 0),
                                  enet_alpha=w.get("enet_alpha", 1.0), audit_bounds=1)
    out = pkg.solve_path(XT, y, ratios, n=w["n"], opts=opts)
    torch.cuda.synchronize()
    st = pkg.stats_to_numpy(out["stats"])
    return {"max_ratio_fp32": float(st["bound_ratio"].max()), "lambdas": int(T),
            "checks": int(st["checks"].sum()),
            "what": "max over all checks and features of |c~_j - x_j^T rho| / E_j, c~ the FP32 correlation "
                    "the safe test uses, x_j^T rho exact (double-float residual, exact sum), E_j its bound"}


def _gpu_sample(pkg, torch, dev, stream, flush, w, XT, y, ratios_h, opts, reps=3):
    """The GPU path on the oracle's sample (the first lambdas of the grid),
    L2 flushed, for a lambda-matched comparison with cpu_baseline."""
    r = torch.from_numpy(ratios_h).to(dev)
    T = len(ratios_h)
    pkg.solve_path(XT, y, r, n=w["n"], opts=opts)
    times, ok = [], 0
    for _ in range(reps):
        flush.fill_(7)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = pkg.solve_path(XT, y, r, n=w["n"], opts=opts)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        ok = int((pkg.stats_to_numpy(out["stats"])["status"] == 0).sum())
    ms = statistics.mean(times)
    return {"value": ok / (ms / 1e3), "unit": "solves/s", "ms": ms, "lambdas": T,
            "sample": f"the same first {T} lambdas on the GPU path (mean of {reps} L2-flushed launches)"}


def _xtr_pass(pkg, torch, dev, stream, flush, peak, peak_src, XT, n, p, ldx, label, reps=10):
    """Event-timed launches of the standalone correlation pass (c = X^T r,
    ||c||_inf), L2 flushed before each; algorithmic bytes = X + r + c.
    The flush writes 512 MiB and then reads 256 MB, so L2 holds clean lines
    when the timed launch starts and none of its DRAM time goes to writing
    back the flush's dirty lines."""
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    r = torch.randn((n,), generator=g, device=dev, dtype=torch.float32)
    c = torch.empty((p,), dtype=torch.float32, device=dev)
    m = torch.empty((1,), dtype=torch.float32, device=dev)
    clean = torch.ones((64 << 20,), dtype=torch.float32, device=dev)
    times = []
    for k in range(3 + reps):
        flush.fill_(k & 0xff)
        clean.sum()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pkg.lasso_correlations_f32(XT.data_ptr(), n, p, ldx, r.data_ptr(), c.data_ptr(), m.data_ptr(),
                                   stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 3:
            times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    nbytes = 4.0 * n * p + 4.0 * n + 4.0 * p
    ach = nbytes / (ms / 1e3) / 1e9
    return {"workload": label, "n": n, "p": p, "bytes_per_launch": nbytes, "ms_per_launch": ms,
            "launches": reps, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
            "l2": "flushed before each launch (512 MiB write, then a 256 MB read)"}


def _tc_gemm(pkg, torch, dev, stream, flush, peaks, n=2000, p=100000, B=1024, reps=5):
    """The batched correlation product of the large multi-RHS design on the
    tensor cores, in the split-BF16 form the lockstep solver runs: K = 3L
    (L = n rounded up to 8) BF16 rows [xh | xh | xl] against [rh | rl | rh].
    Executed flops are 2 (3L) p B; the method's flops (one product X^T R) are
    2 n p B.  L2 flushed before each launch."""
    L = (n + 7) // 8 * 8
    K = 3 * L
    g = torch.Generator(device=dev)
    g.manual_seed(11)
    Xb = torch.randn((p, K), generator=g, device=dev, dtype=torch.float32).to(torch.bfloat16)
    Rb = torch.randn((B, K), generator=g, device=dev, dtype=torch.float32).to(torch.bfloat16)
    C = torch.empty((B, p), dtype=torch.float32, device=dev)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    times = []
    for k in range(2 + reps):
        flush.fill_(k & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pkg.lasso_correlations_bf16(Xb.data_ptr(), K, p, K, Rb.data_ptr(), K, B, C.data_ptr(), p, ws.data_ptr(), 256,
                                    stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    ex = 2.0 * K * p * B / (ms / 1e3) / 1e12
    me = 2.0 * n * p * B / (ms / 1e3) / 1e12
    peak = peaks.get("bf16_tflops")
    del Xb, Rb, C
    return {"workload": f"split-BF16 X^T R, n={n} (K=3L={K}), p={p}, B={B}", "ms_per_launch": ms,
            "executed_tflops": ex, "method_tflops": me, "peak_bf16_tflops": peak,
            "frac_executed": ex / peak if peak else None,
            "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)" if peak else "none",
            "l2": "flushed before each launch"}


def _tuned_vs_plain(pkg, torch, dev, stream, flush, sample):
    """Stability-selection workload (256 row-subset problems, 50 lambdas):
    the batched solver in both modes against the plain single-problem path run
    one problem at a time on a bounded sample."""
    import numpy as np
    import gen
    w = gen.workload3()
    n, p, B, T = w["n"], w["p"], w["Y"].shape[0], w["T"]
    XT = torch.from_numpy(w["XT"]).to(dev)
    Y = torch.from_numpy(w["Y"]).to(dev)
    M = torch.from_numpy(w["row_mask"]).to(dev)
    ratios = torch.from_numpy(pkg.lasso_lambda_grid(T, w["delta"])).to(dev)
    out = {"workload": w["name"] + ": Gaussian 1000x20000 FP32, 256 row subsets of U{400..1000}, beta* 30-sparse, "
           "SNR 5, T=50 to lambda_max/100, check every 10 passes, gap<=1e-6*||y||^2", "problems": B, "T": T}
    launches = 0
    for name, gd in (("batched_fp32", pkg.LASSO_F32), ("batched_split_bf16_tc", pkg.LASSO_BF16)):
        opts = pkg.lasso_default_opts(xtr_scope=1, gemm_dtype=gd, screen_period=w["f"], gap_tol_rel=w["tol"])
        pkg.solve_batch(XT, Y[:8].contiguous(), ratios, n=n, row_mask=M[:8].contiguous(), opts=opts)
        torch.cuda.synchronize()
        flush.fill_(3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = pkg.solve_batch(XT, Y, ratios, n=n, row_mask=M, opts=opts)
        e1.record(stream)
        torch.cuda.synchronize()
        st = pkg.stats_to_numpy(res["stats"])
        ok = int((st["status"] == 0).sum())
        ms = e0.elapsed_time(e1)
        out[name] = {"solves_per_s": ok / (ms / 1e3), "certified": ok, "solves": B * T, "ms": ms}
        del res
    # plain: lasso_path per problem on its gathered rows (X restricted, ld a multiple of 4)
    opts = pkg.lasso_default_opts(screen_period=w["f"], gap_tol_rel=w["tol"])
    tot_ms, tot_ok = 0.0, 0
    for b in range(-1, sample):
        bb = max(b, 0)
        rows = np.nonzero(w["row_mask"][bb])[0]
        m = rows.size
        ld = (m + 3) // 4 * 4
        Xb = torch.zeros((p, ld), dtype=torch.float32, device=dev)
        Xb[:, :m] = XT[:, torch.from_numpy(rows).to(dev)]
        yb = torch.from_numpy(np.ascontiguousarray(w["Y"][bb, rows])).to(dev)
        flush.fill_(5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = pkg.solve_path(Xb, yb, ratios, n=m, opts=opts)
        e1.record(stream)
        torch.cuda.synchronize()
        if b >= 0:  # b = -1 is the untimed warm-up
            st = pkg.stats_to_numpy(res["stats"])
            tot_ok += int((st["status"] == 0).sum())
            tot_ms += e0.elapsed_time(e1)
    out["plain_single_path"] = {"solves_per_s": tot_ok / (tot_ms / 1e3), "certified": tot_ok,
                                "solves": sample * T, "ms": tot_ms,
                                "sample": f"first {sample} of the {B} problems, one lasso_path call each"}
    # row a11 on the tensor-core path: one untimed audited lockstep run on a sample
    opts = pkg.lasso_default_opts(xtr_scope=1, gemm_dtype=pkg.LASSO_BF16, screen_period=w["f"], gap_tol_rel=w["tol"],
                                  audit_bounds=1)
    aud = pkg.solve_batch(XT, Y[:32].contiguous(), ratios, n=n, row_mask=M[:32].contiguous(), opts=opts)
    torch.cuda.synchronize()
    sa = pkg.stats_to_numpy(aud["stats"])
    out["bound_audit"] = {"problems": 32, "lambdas": T, "max_ratio_split_bf16_tc": float(sa["bound_ratio_tc"].max()),
                          "max_ratio_fp32": float(sa["bound_ratio"].max()),
                          "what": "max |c~_j - x_j^T rho| / E_j: first checks from the split-BF16 tensor-core "
                                  "product (tc), later checks FP32 CUDA-core dots"}
    del aud
    best = max(out["batched_fp32"]["solves_per_s"], out["batched_split_bf16_tc"]["solves_per_s"])
    out["tuned_over_plain"] = best / out["plain_single_path"]["solves_per_s"]
    out["note"] = ("tuned = batched persistent CD (one CTA per problem) with the tensor-core split-BF16 first "
                   "check or FP32 checks, best of the two; plain = the single-problem path")
    return out


def _tuned_vs_plain_large(pkg, torch, dev, stream, flush, B, plain=2):
    """The metric's large configuration: Gaussian 2000 x 100000 FP32 (800 MB),
    right-hand sides with beta* sparsity k ~ U{10..200} and SNR ~ U[1,10],
    30 lambdas to lambda_max/100.  Tuned: the batched solver with the launch
    shape lasso_batch_tune picks (split-BF16 tensor-core first checks or FP32
    checks, CTAs per problem) on the first B right-hand sides; plain: the single
    path per right-hand side on the first `plain` of them.  The learned start is
    not part of this line (its network at this design size is p x n = 2e8
    parameters); the 300 x 10000 learned line measures it."""
    import numpy as np
    import gen
    w = gen.workload5()
    n, p, T = w["n"], w["p"], w["T"]
    XT = torch.from_numpy(w["XT"]).to(dev)
    Y = torch.from_numpy(np.ascontiguousarray(w["Y"][:B])).to(dev)
    ratios = torch.from_numpy(pkg.lasso_lambda_grid(T, w["delta"])).to(dev)
    base = dict(screen_period=w["f"], gap_tol_rel=w["tol"])
    tuned, times = pkg.tune_batch(XT, Y, ratios, n=n, opts=pkg.lasso_default_opts(**base),
                                  sample=min(B, 32), lambdas=3)
    torch.cuda.synchronize()
    flush.fill_(9)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = pkg.solve_batch(XT, Y, ratios, n=n, opts=tuned)
    e1.record(stream)
    torch.cuda.synchronize()
    st = pkg.stats_to_numpy(res["stats"])
    ok = int((st["status"] == 0).sum())
    ms = e0.elapsed_time(e1)
    del res
    pms, pok = 0.0, 0
    popts = pkg.lasso_default_opts(**base)
    for b in range(-1, plain):
        yb = torch.from_numpy(np.ascontiguousarray(w["Y"][max(b, 0)])).to(dev)
        flush.fill_(10)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = pkg.solve_path(XT, yb, ratios, n=n, opts=popts)
        e1.record(stream)
        torch.cuda.synchronize()
        if b >= 0:
            pms += e0.elapsed_time(e1)
            pok += int((pkg.stats_to_numpy(out["stats"])["status"] == 0).sum())
    del XT
    tuned_sps = ok / (ms / 1e3)
    plain_sps = pok / (pms / 1e3)
    shape = {"gemm_dtype": "split_bf16_tc" if tuned.gemm_dtype == pkg.LASSO_BF16 else "fp32",
             "batch_ctas_per_sm": int(tuned.batch_ctas_per_sm), "gemm_tile_n": int(tuned.gemm_tile_n),
             "batch_group": int(tuned.batch_group), "lockstep_pass": int(tuned.lockstep_pass)}
    return {"workload": w["name"] + ": Gaussian 2000x100000 FP32, k~U{10..200}, SNR~U[1,10], T=30 to "
                                    "lambda_max/100, check every 10 passes, gap<=1e-6*||y||^2",
            "tuned": {"solves_per_s": tuned_sps, "certified": ok, "solves": B * T, "ms": ms,
                      "sample": f"first {B} of the 1024 right-hand sides, one lasso_batch call",
                      "launch_shape": shape, "shape_times_ms": [float(x) for x in times]},
            "plain_single_path": {"solves_per_s": plain_sps, "certified": pok, "solves": plain * T, "ms": pms,
                                  "sample": f"first {plain} right-hand sides, one lasso_path call each"},
            "tuned_over_plain": tuned_sps / plain_sps if plain_sps > 0 else None,
            "target": ">= 5x with learned start + batched + mixed precision",
            "note": "bounded sample of the 1024 right-hand sides so that the default bench ends in minutes (a "
                    "sample this small leaves most SMs idle in the batched solver; --large-sample 304 runs one "
                    "resident wave); the learned start is measured on the 300 x 10000 workload"}


def _learned(pkg, torch, dev, stream, n_train, epochs=20, lr=1e-2, n_eval=1024):
    """Learned warm start on the fixed 300 x 10000 design at lambda =
    lambda_max / 20: solver solutions of n_train responses train the 8-layer
    net (hand-written forward/backward/Adam kernels); held-out responses are
    then solved from the zero start and from the net's beta0."""
    import numpy as np
    import gen
    w = gen.workload4()
    n, p = w["n"], w["p"]
    XT = torch.from_numpy(w["XT"]).to(dev)
    ratio = torch.tensor([w["lambda_ratio"]], dtype=torch.float64, device=dev)
    opts = pkg.lasso_default_opts(gemm_dtype=pkg.LASSO_F32)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    Ytr = torch.from_numpy(w["sample"](n_train, 1)).to(dev)
    Yev = torch.from_numpy(w["sample"](n_eval, 2)).to(dev)
    tr, ms_gen = timed(lambda: pkg.solve_batch(XT, Ytr, ratio, n=n, opts=opts))
    net = pkg.ListaNet(XT, n, L=8, ratio=w["lambda_ratio"])
    Ytil, s = net.normalize(Ytr)
    tgt = net.targets(tr["beta"][:, 0, :].contiguous(), s)
    del tr
    hist, ms_train = timed(lambda: net.fit(Ytil, tgt, epochs=epochs, batch=256, lr=lr, seed=7))
    pkg.solve_batch(XT, Yev[:8].contiguous(), ratio, n=n, opts=opts)
    z, ms_zero = timed(lambda: pkg.solve_batch(XT, Yev, ratio, n=n, opts=opts))
    b0, ms_net = timed(lambda: net.warm_start(Yev))
    wres, ms_warm = timed(lambda: pkg.solve_batch(XT, Yev, ratio, n=n, beta0=b0, opts=opts))
    s0 = pkg.stats_to_numpy(z["stats"])
    s1 = pkg.stats_to_numpy(wres["stats"])
    bz = z["beta"][:, 0, :]
    rel = (torch.linalg.norm(b0 - bz, dim=1) / torch.linalg.norm(bz, dim=1).clamp_min(1e-300)).cpu().numpy()
    return {"workload": w["name"] + ": Gaussian 300x10000 FP32, k~U{5..50}, SNR~U[2,10], lambda=lambda_max/20",
            "n_train": n_train, "n_eval": n_eval, "epochs": epochs, "lr_relative": lr,
            "ms_generate_targets": ms_gen, "ms_train": ms_train, "loss_first_epoch": hist[0],
            "loss_last_epoch": hist[-1],
            "zero_start": {"solves_per_s": int((s0["status"] == 0).sum()) / (ms_zero / 1e3), "ms": ms_zero,
                           "mean_passes": float(s0["epochs"].mean()), "x_columns": int(s0["x_columns"].sum())},
            "learned_start": {"solves_per_s": int((s1["status"] == 0).sum()) / ((ms_warm + ms_net) / 1e3),
                              "ms": ms_warm, "ms_net": ms_net, "mean_passes": float(s1["epochs"].mean()),
                              "x_columns": int(s1["x_columns"].sum())},
            "beta0_rel_err_median": float(np.median(rel))}


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
