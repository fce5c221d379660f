#!/usr/bin/env python
"""Benchmark of the line-by-line emission model on GB300.

One step = one HMC-style forward + gradient of the 100-layer emission model:
layer temperatures, both species' line-sum cross-sections, optical depth,
emission solve, Gaussian log-likelihood, and the adjoints of all of them, in the
mixed precision form (FP32 Voigt and compensated sums, FP64 offsets and
strengths, FP64 radiative transfer).  The metric counts Voigt evaluations: every
in-cut (line, grid point, layer) triple is evaluated once in the forward line sum
and once in its adjoint.

The headline workload is the precision form at scale: 10,000,000 water-like +
200,000 CO-like lines, a 100,000-point log grid over 4340-4390 cm^-1, 100 layers
(1e-3 .. 1e2 bar), W = 25 cm^-1.  The emission workload (200,000 + 20,000 lines,
20,000 points) is timed beside it under "extra".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica (its own theta);
there is no data-path collective (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

T_START = time.perf_counter()
# the whole command must end well inside the caller's limit (1,800 s): optional
# legs are skipped, and say so, once the run gets near this budget
WALL_BUDGET_S = 1600.0

FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM on sm_103a (one FFMA = 2 flops)

# FP32 flops per in-cut triple of the two line-sum kernels, from the SASS
# instruction counts of one ncu capture per workload (FFMA 2, FADD/FMUL 1, packed
# FFMA2 4, FADD2/FMUL2 2 flops per thread instruction; MUFU reciprocals not
# counted), divided by the launch's in-cut triples.  Valid only for the kernel
# sources they were taken on (the hash); otherwise the bench falls back to the
# cheapest-form lower bound and says so.
FLOPS_PER_TRIPLE = {
    "sources_sha256": "bcfd701beb7a1f40c608e700fbcde5e1301ffb6eae228c6aed4523b1b23de8d7",
    "scale": {"fwd": 9.00, "adj": 13.21,
              "capture": "both species' launches of a 5-layer slice of the 10.2M-line workload (10,000,000 + "
                         "200,000 lines, 100,000 points): 3.44e13 and 5.05e13 FP32 flops over 3.82e12 triples"},
    "emission": {"fwd": 9.16, "adj": 13.38,
                 "capture": "both species' launches of a 20-layer slice of the emission workload (200,000 + 20,000 "
                            "lines, 20,000 points): 6.05e11 and 8.84e11 FP32 flops over 6.60e10 triples"},
}
FLOPS_LOWER_BOUND = {"fwd": 8, "adj": 12}  # cheapest packed wing forms, RCP counted as 1 flop

# DRAM bytes (read + write) per layer of one launch of each line-sum kernel, averaged
# over the two species' launches, from one ncu capture of the same reduced-layer
# slices (the traffic is per layer: each layer's records are read once from DRAM
# when L2 serves the re-reads); null unless the sources still hash to the captured ones.
TRAFFIC = {
    "sources_sha256": "bcfd701beb7a1f40c608e700fbcde5e1301ffb6eae228c6aed4523b1b23de8d7",
    "scale": {"fwd": 2.992e8, "adj": 3.132e8},
    "emission": {"fwd": 3.04e7, "adj": 5.76e7},
    "capture": "ncu dram__bytes_read.sum + dram__bytes_write.sum of both species' launches, 5-layer slice of the "
               "10.2M-line workload and 20-layer slice of the emission workload, scaled to the launch's layers",
}


def kernel_sources_sha256():
    h = hashlib.sha256()
    for f in ("xs_linesum.cu", "xs_device.cuh"):
        with open(os.path.join(ROOT, "paper_2105_14782_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def elapsed():
    return time.perf_counter() - T_START


def job_throughput(ms_local, evals_per_step, steps, world, dist=None, device="cpu"):
    """Whole-job time and throughput of `world` replicas: the slowest rank's time
    (max over ranks) and the evaluations of all ranks over it."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    return t_max, world * evals_per_step * steps / (t_max / 1000.0)


def in_cut_counts(lines, nu, W_cut):
    """In-cut lines per grid point (every layer has the same cut)."""
    c = np.sort(lines.nu_hat)
    return np.searchsorted(c, nu + W_cut, side="right") - np.searchsorted(c, nu - W_cut, side="left")


def in_cut_triples(lines, nu, W_cut, L):
    return int(np.sum(in_cut_counts(lines, nu, W_cut))) * L


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


WORKLOAD_TEXT = {
    "scale": "precision form at scale: 100 layers 1e-3..1e2 bar, 10,000,000 water-like + 200,000 CO-like lines, "
             "100,000-point log grid 4340-4390 cm^-1, W = 25 cm^-1",
    "emission": "emission: 100 layers 1e-3..1e2 bar, 200,000 water-like + 20,000 CO-like lines, 20,000-point log "
                "grid 4340-4390 cm^-1, W = 25 cm^-1",
}


def atmosphere(name, n_layers=100):
    if name == "emission":
        return W.emission_case(n_layers=n_layers)
    cfg = W.WORKLOADS["scale"]
    p, dp = W.pressure_layers(n_layers)
    return W.Atmosphere(species=[W.water_like(cfg["n_water"]), W.co_like(cfg["n_co"])], vmr=[1e-3, 5e-4],
                        nu=W.grid_lognu(cfg["n_grid"]), p_bar=p, dp_bar=dp)


class ClockSampler:
    """nvidia-smi samples of SM clock, power and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, pw, mx, reasons = [], [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
                pw.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_median": statistics.median(pw) if pw else None}


# ------------------------------------------------------------------ oracle legs (CPU)


def oracle_pair_rate(species, nu, T, P, layer, gi, wing_cut=25.0):
    """Oracle line sums at grid points gi of one layer, all species.  The oracle
    first derives every line's parameters for the layer (one pass over the list);
    that setup is timed on a call with no points and subtracted, so the rate is
    that of the line sums themselves.  Returns (evaluations, seconds)."""
    import oracle
    ev, dt = 0, 0.0
    li = np.zeros(gi.size, dtype=np.int32)
    none_l, none_g = np.zeros(0, dtype=np.int32), np.zeros(0, dtype=np.int64)
    for sp in species:
        t0 = time.perf_counter()
        oracle.xs_points(sp, nu, T[layer:layer + 1], P[layer:layer + 1], none_l, none_g, wing_cut=wing_cut)
        t1 = time.perf_counter()
        oracle.xs_points(sp, nu, T[layer:layer + 1], P[layer:layer + 1], li, gi, wing_cut=wing_cut)
        t2 = time.perf_counter()
        ev += int(in_cut_counts(sp, nu[gi], wing_cut).sum())
        dt += max((t2 - t1) - (t1 - t0), 1e-9)
    return ev, dt


def cpu_baseline(atm, budget_s=15.0, seed=0):
    """The FP64 oracle on a bounded sample of the same workload: random grid points
    of one random layer, all species, on every host core; evaluations counted per
    sampled point.  The sample holds at least 64 points so that the oracle's
    parallel loop over points keeps every core busy."""
    import oracle
    rng = np.random.default_rng(W.SEED_SUBSET + 100 + seed)
    T = W.THETA_STAR[0] * atm.p_bar ** W.THETA_STAR[1]
    L, N = len(atm.p_bar), len(atm.nu)
    per_point = sum(float(np.mean(in_cut_counts(sp, atm.nu, atm.wing_cut))) for sp in atm.species)
    n_pts = int(max(64, min(20000, budget_s * 5e7 / per_point)))  # sized for ~5e7 evaluations/s
    layer = int(rng.integers(L))
    ev, dt = oracle_pair_rate(atm.species, atm.nu, T, atm.p_bar, layer, np.sort(rng.integers(0, N, n_pts)))
    return {"value": ev / dt, "unit": "evals/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle forward line sums at {n_pts} random grid points of layer {layer}, all species "
                      f"({ev:.3g} Voigt evaluations, {dt:.1f} s of line sums; the layer's one-pass line-parameter "
                      "setup timed on a call with no points and excluded)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    atm = atmosphere(args.workload)
    for i in range(args.warmup):
        cpu_baseline(atm, budget_s=2.0, seed=1000 + i)
    vals = []
    t0 = time.perf_counter()
    last = None
    for i in range(args.steps):
        last = cpu_baseline(atm, budget_s=8.0, seed=i)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": "Voigt line x grid x layer evals/s", "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload],
                       "sample": "each step: oracle forward line sums at random grid points of one random layer"},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU legs


def timed_ms(fn, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    r = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b), r


def error_block(dev, atm, model, theta, stream):
    """Relative error of the mixed path against the FP64 GPU path on the same GPU,
    per result, at theta:
      sigma: every layer at a block of 256 consecutive grid points (seeded start),
             both species, where sigma > 1e-6 of the layer maximum; the mixed values
             come from the full-grid call in the step's launch configuration;
      F0:    the model's spectrum at those points against the FP64 line sums
             composed with the FP64 optical depth and emission solve;
      gradient: logL over a 64-point window and its gradient, mixed vs FP64."""
    import torch
    from paper_2105_14782_gb300 import xs
    f64 = dict(dtype=torch.float64, device=dev)
    N, L = len(atm.nu), len(atm.p_bar)
    rng = np.random.default_rng(W.SEED_SUBSET + 7)
    j0 = int(rng.integers(0, N - 256))
    blk = np.arange(j0, j0 + 256)
    T = xs.layer_temperatures(theta[0], theta[1], model.P)
    sb = float(theta[-1])
    nu_b = torch.as_tensor(atm.nu[blk], **f64)
    out, s64s = {}, []
    worst, ms64, ev64 = 0.0, 0.0, 0
    for k, dl in enumerate(model.species):
        smx = xs.xs_compute(dl, model.nu, T, model.P, broad_scale=sb, wing_cut=atm.wing_cut, prec=xs.PREC_MIXED,
                            workspace=model.ws)[:, blk].double()
        ms, s64 = timed_ms(lambda: xs.xs_compute(dl, nu_b, T, model.P, broad_scale=sb, wing_cut=atm.wing_cut,
                                                 prec=xs.PREC_FP64), stream)
        ms64 += ms
        ev64 += int(in_cut_counts(atm.species[k], atm.nu[blk], atm.wing_cut).sum()) * L
        m = s64 > 1e-6 * s64.max(dim=1, keepdim=True).values
        worst = max(worst, float(((smx - s64).abs() / s64)[m].max()))
        s64s.append(s64)
    out["sigma_max_rel"] = worst
    S = len(model.species)
    vmr = torch.as_tensor(np.array([[10.0 ** theta[2 + m]] * L for m in range(S)]), **f64)
    dtau = xs.tau_layers(s64s, vmr, model.P, model.dP, atm.gravity, atm.mu, atm.kappa_coef, prec=xs.PREC_FP64)
    F64 = xs.emission_spectrum(dtau, T, nu_b)
    Fmx = model.F0[torch.as_tensor(blk, device=dev)]  # the spectrum of the last end-to-end step, at theta
    out["F0_max_rel"] = float(((Fmx - F64).abs() / F64).max())
    # gradient of logL over a 64-point window
    w = blk[:64]
    sub = W.Atmosphere(species=atm.species, vmr=atm.vmr, nu=atm.nu[w], p_bar=atm.p_bar, dp_bar=atm.dp_bar,
                       wing_cut=atm.wing_cut, kappa_coef=atm.kappa_coef, gravity=atm.gravity, mu=atm.mu)
    d_w, s_w = model.d_obs.cpu().numpy()[w], model.sig_obs.cpu().numpy()[w]
    g = {}
    for name, prec in (("mixed", xs.PREC_MIXED), ("fp64", xs.PREC_FP64)):
        m = xs.EmissionModel(sub, prec=prec, device=dev, lines=model.species, d_obs=d_w, sig_obs=s_w)
        g[name] = m.logl_grad_async(theta).cpu().numpy()
        del m
        torch.cuda.empty_cache()
    rel = np.abs(g["mixed"] - g["fp64"]) / np.abs(g["fp64"])
    out["logL_rel"] = float(rel[0])
    out["grad_max_rel"] = float(rel[1:].max())
    out["grad_rel"] = [float(v) for v in rel[1:]]
    out["where"] = (f"sigma and F0: all {L} layers x grid points {j0}..{j0 + 255}; gradient: logL over grid "
                    f"points {j0}..{j0 + 63}, theta = {[round(float(v), 4) for v in theta]}")
    out["tolerance"] = {"sigma": 1e-5, "F0": 1e-6, "grad": 1e-4}
    torch.cuda.empty_cache()
    fp64 = {"forward_ms_256_points": ms64, "forward_evals_per_s": ev64 / (ms64 / 1000.0)}
    return out, fp64


def step_bench(dev, stream, atm, prec, steps, warmup, rank, world, dist, e2e_steps):
    """Warm up, time `steps` forward + gradient steps (CUDA events on the launching
    stream, barrier and synchronize on both sides), then the end-to-end steps."""
    import torch
    from paper_2105_14782_gb300 import xs
    L, N = len(atm.p_bar), len(atm.nu)
    triples = sum(in_cut_triples(sp, atm.nu, atm.wing_cut, L) for sp in atm.species)
    model = xs.EmissionModel(atm, prec=prec, device=dev)
    F_star = model.forward(W.THETA_STAR).clone()
    sig = 0.01 * F_star
    model.set_observation(F_star + sig * torch.as_tensor(W.std_normal(N), device=dev), sig)
    theta = W.theta_points(64)[rank % 64]
    for _ in range(warmup):
        model.logl_grad_async(theta)
    torch.cuda.synchronize(dev)

    gpu_index = int(os.environ.get("LOCAL_RANK", "0"))
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        gpu_index = vis.split(",")[gpu_index]
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.5)
    xs.profile(True)
    n0 = xs.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        model.logl_grad_async(theta)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = (xs.launch_count() - n0) / steps
    prof = xs.profile_read()
    xs.profile(False)
    clk = clocks.stop()
    assert np.all(np.isfinite(model.out.cpu().numpy())), "non-finite logL or gradient"
    evals_per_step = 2 * triples
    t_max, value = job_throughput(ms, evals_per_step, steps, world, dist, dev)

    # end to end through the public API with host buffers: line lists, grid, layers
    # and the observed spectrum go host -> device every step; logL, gradient and the
    # spectrum come back
    host = [[t.cpu().pin_memory() for t in sp.tensors] for sp in model.species]
    host_misc = [x.cpu().pin_memory() for x in (model.nu, model.P, model.dP, model.d_obs, model.sig_obs)]
    out_h = torch.empty(model.out.shape, dtype=torch.float64).pin_memory()
    F_h = torch.empty(N, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * 8 for sp in host for t in sp) + sum(x.numel() * 8 for x in host_misc)
    d2h = out_h.numel() * 8 + F_h.numel() * 8

    def e2e_step():
        for sp, hs in zip(model.species, host):
            for dt_, ht in zip(sp.tensors, hs):
                dt_.copy_(ht, non_blocking=True)
        for dt_, ht in zip((model.nu, model.P, model.dP, model.d_obs, model.sig_obs), host_misc):
            dt_.copy_(ht, non_blocking=True)
        model.logl_grad_async(theta, F0=model.F0)
        out_h.copy_(model.out, non_blocking=True)
        F_h.copy_(model.F0, non_blocking=True)

    if ms / steps > 10000.0:
        e2e_steps = 1  # a step of tens of seconds: one end-to-end step keeps the run inside its time limit
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    b.record(stream)
    torch.cuda.synchronize(dev)
    e_ms = a.elapsed_time(b) / e2e_steps
    assert np.all(np.isfinite(out_h.numpy())), "non-finite end-to-end result"
    e2e = {"value": world * evals_per_step / (e_ms / 1000.0), "unit": "evals/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e_ms, "steps": e2e_steps}
    return dict(model=model, theta=theta, triples=triples, evals_per_step=evals_per_step, ms=ms, t_max=t_max,
                value=value, launches=launches, prof=prof, clocks=clk, e2e=e2e)


def roofline(res, atm, workload, steps, n_sm, clk):
    """The dominant line-sum kernel against the FP32 pipe: FP32 flops per launch
    (flops per in-cut triple x the launch's triples) over its mean launch time."""
    fwd_ms, fwd_n, adj_ms, adj_n = res["prof"]
    kind = "adj" if adj_ms >= fwd_ms else "fwd"
    k_ms = (adj_ms if kind == "adj" else fwd_ms) / max(adj_n if kind == "adj" else fwd_n, 1)
    per_launch = res["triples"] / len(atm.species)  # one launch per species and step, averaged over species
    fl = FLOPS_PER_TRIPLE.get(workload)
    measured = bool(fl) and FLOPS_PER_TRIPLE["sources_sha256"] == kernel_sources_sha256()
    fpt = fl[kind] if measured else FLOPS_LOWER_BOUND[kind]
    achieved = per_launch * fpt / (k_ms / 1000.0) / 1e12
    peaks = read_peaks()
    sm_max = float(clk.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0)
    peak_max = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    sm_med = clk.get("sm_mhz") or sm_max
    peak_med = n_sm * FP32_LANES_PER_SM * 2 * sm_med * 1e6 / 1e12
    traffic = None
    if TRAFFIC["sources_sha256"] == kernel_sources_sha256() and TRAFFIC.get(workload):
        traffic = TRAFFIC[workload][kind] * len(atm.p_bar)
    # algorithmic bytes of one launch (averaged over species): per (layer, line) the
    # records rec1 + rec2 + near range (+ rec3 in the adjoint), per line the cut range
    # and centre pair, per layer and point the lambda or near-sum read and the output
    L, N = len(atm.p_bar), len(atm.nu)
    nl_avg = sum(sp.n for sp in atm.species) / len(atm.species)
    rec = 48 if kind == "adj" else 40
    algo_bytes = nl_avg * (rec * L + 16) + L * N * (8 + (0 if kind == "adj" else 4))
    name = "linesum_adjoint_kernel<float>" if kind == "adj" else "linesum_kernel<float>"
    return {"bound": "alu", "achieved": achieved, "peak": peak_max, "unit": "TFLOP/s", "frac": achieved / peak_max,
            "traffic": traffic, "kernel": name, "kernel_ms_per_launch": k_ms, "triples_per_launch": per_launch,
            "flops_per_triple": fpt,
            "flops_basis": (f"ncu SASS FP32 instruction counts ({fl['capture']})" if measured else
                            "lower bound: cheapest packed wing form, ncu counts not taken on these sources"),
            "peak_note": f"FP32 pipe: {n_sm} SMs (device) x {FP32_LANES_PER_SM} lanes x 2 flop x {sm_max:.0f} MHz "
                         "(max SM clock); derived, not measured",
            "frac_at_sampled_clock": achieved / peak_med, "sampled_sm_mhz": sm_med,
            "algorithmic_bytes": algo_bytes,
            "traffic_note": TRAFFIC["capture"] if traffic else "no ncu DRAM capture on these sources"}


def serving(dev, budget_s):
    """Continuous-batching server under the HMC request mix (256 chains, 200 req/s
    offered; line count log-uniform 1e3..1e6, grid 2,000..50,000, layers 20..200):
    a saturated closed loop (the saturation point), then open-loop Poisson
    arrivals at two fractions of the capacity it measured, each until at least
    300 requests have completed, with latency binned by request size, the FP64
    path on a bounded sample of the same stream, and a burst of MODIT requests."""
    import torch
    from paper_2105_14782_gb300 import serve, xs

    t_setup = time.perf_counter()
    pool = serve.LinePool(dev)
    mean_ev = serve.mean_request_evals(pool)
    arena_bytes, slots = 64 << 30, 4
    sched, _ = serve.make_server(arena_bytes=arena_bytes, slots=slots, pool=pool, device=dev, priority=True,
                                 hi_evals=1e11)
    warm = serve.request_stream(8, seed=W.SEED_SERVE + 50)
    for r in warm:
        r.n_lines, r.n_grid = 1000, 2000
        sched.submit(r)
    sched.drain(timeout_s=120)
    setup_s = time.perf_counter() - t_setup

    fin, wall = serve.closed_loop(sched, chains=256, offered_rate=200.0, duration_s=15.0, cancel_at_end=True)
    closed = serve.summarize(fin, wall)
    closed.update(chains=256, offered_req_per_s=200.0, window_s=15.0,
                  note="saturated: 200 req/s offered against a capacity of a few req/s; its latencies are queueing "
                       "under overload, not a sustained p99")
    cap = closed["evals_per_s"] / mean_ev
    slo = 4.0
    points = []
    for frac in (0.8, 0.5):
        need_s = 330.0 / (frac * cap) + 5.0
        if elapsed() + need_s > budget_s:
            points.append({"load_fraction": frac, "skipped": f"time budget ({need_s:.0f} s needed)"})
            continue
        s2 = serve.Scheduler(sched.ex, arena_bytes, slots)
        sent, wall2 = serve.open_loop(s2, rate=frac * cap, duration_s=need_s - 5.0, seed=W.SEED_SERVE + int(frac * 10))
        st = serve.summarize(sent, wall2)
        st.update(load_fraction=frac, offered_req_per_s=frac * cap, window_s=need_s - 5.0,
                  by_size=serve.latency_by_size(sent), slo_met=st["p99_s"] <= slo)
        points.append(st)
    sample = [r for r in serve.request_stream(400, seed=W.SEED_SERVE + 1)
              if 2 * r.n_layers * r.n_grid * r.n_lines * 0.75 <= 2e10][:6]
    res = {}
    for prec in (xs.PREC_MIXED, xs.PREC_FP64):
        ex = serve.LibxsExecutor(pool, sched.ex.arena_t, sched.ex.streams, prec=prec)
        s1 = serve.Scheduler(ex, arena_bytes, 1)
        reqs = [serve.Request(rid=r.rid, chain=0, n_lines=r.n_lines, n_grid=r.n_grid, n_layers=r.n_layers,
                              theta=r.theta) for r in sample]
        t0 = time.perf_counter()
        for r in reqs:
            s1.submit(r)
            s1.drain(timeout_s=300)
        dt = time.perf_counter() - t0
        assert all(r.status == serve.DONE for r in reqs)
        res[prec] = (sum(r.evals for r in reqs) / dt, [r.latency for r in reqs])
    e64, lat64 = res[xs.PREC_FP64]
    emx, latmx = res[xs.PREC_MIXED]
    modit = None
    if elapsed() + 60.0 < budget_s:
        try:
            modit = modit_burst(sched, arena_bytes, slots)
        except Exception as e:  # reported, not fatal to the line
            modit = {"error": f"{type(e).__name__}: {e}"}
    fp64 = {"evals_per_s": e64, "capacity_req_per_s": e64 / mean_ev, "latency_s": lat64,
            "mixed_evals_per_s_same_requests": emx, "mixed_latency_s": latmx,
            "sample": f"{len(sample)} requests of the stream with <= 2e10 evaluations each, run one at a time"}
    del sched, pool
    torch.cuda.empty_cache()
    return {"slo_p99_s": slo, "open_loop": points, "closed_loop_saturation": closed, "capacity_req_per_s": cap,
            "mean_request_evals": mean_ev, "fp64_path": fp64, "modit_burst": modit, "slots": slots,
            "arena_bytes": arena_bytes,
            "setup_s": setup_s,
            "priority": "line-sum requests under 1e11 evaluations run on high-priority streams",
            "requests": "line count log-uniform 1e3..1e6 (served by the nearest of 7 resident water-like lists "
                        "1e3..1e6 plus 2,000 CO-like lines), grid 2,000..50,000, layers 20..200; "
                        "fwd + grad (logL, dlogL/dtheta), FP32 Voigt with FP64 offsets",
            "latency": "submit to result on the host (pinned D2H of logL and gradient done)"}


def modit_burst(sched, arena_bytes, slots, n=100):
    """n requests of the serving stream asking for MODIT, submitted at once to a
    server with the same executor; those whose grid does not resolve the Doppler
    width are rejected at admission.  Latencies of the completed ones."""
    from paper_2105_14782_gb300 import serve
    s3 = serve.Scheduler(sched.ex, arena_bytes, slots)
    mreqs = serve.request_stream(n, seed=W.SEED_SERVE + 60)
    t0 = time.perf_counter()
    for r in mreqs:
        r.method = "modit"
        s3.submit(r)
    s3.drain(timeout_s=600)
    wall = time.perf_counter() - t0
    ok = [r for r in mreqs if r.status == serve.DONE]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
    return {"submitted": len(mreqs), "completed": len(ok),
            "rejected_coarse_grid": sum(r.status == serve.REJECTED and "too coarse" in r.error for r in mreqs),
            "rejected_other": sum(r.status == serve.REJECTED and "too coarse" not in r.error for r in mreqs),
            "failed": sum(r.status == serve.FAILED for r in mreqs), "wall_s": wall,
            "req_per_s": len(ok) / wall, "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "grid_points_completed": [min((r.n_grid for r in ok), default=0), max((r.n_grid for r in ok), default=0)],
            "rule": f"beta' >= {serve.MODIT_MIN_BETA_Q} q steps for every species in the coolest layer",
            "n_gamma": sched.ex.n_gamma,
            "latency": "all submitted at once: latencies include queueing behind the burst"}


def modit_stats(dev, atm):
    """MODIT (Sec. 2.1.2) cross-sections of both species over all layers at theta*,
    FP64 and FP32, against the line-by-line sum (mixed, W = 25 cm^-1) where that is
    above 1e-3 of its layer maximum, and the forward + gradient step on MODIT."""
    import torch
    from paper_2105_14782_gb300 import xs

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            r = fn()
        b.record()
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps, r

    f64 = dict(dtype=torch.float64, device=dev)
    P = torch.as_tensor(atm.p_bar, **f64)
    T = torch.as_tensor(W.THETA_STAR[0] * atm.p_bar ** W.THETA_STAR[1], **f64)
    nu = torch.as_tensor(atm.nu, **f64)
    nu_min, nu_max, N = float(atm.nu[0]), float(atm.nu[-1]), len(atm.nu)
    res = {"n_gamma": 16, "layers": len(atm.p_bar), "grid": N}
    lines = [xs.DeviceLines(sp, dev) for sp in atm.species]
    res["lines"] = [dl.n for dl in lines]
    res["n_fft"] = [xs.modit_fft_length(nu_min, nu_max, N, dl) for dl in lines]
    out = {}
    for name, prec in (("fp64", xs.PREC_FP64), ("fp32", xs.PREC_MIXED)):
        ms = 0.0
        sig = []
        for dl, nf in zip(lines, res["n_fft"]):
            ws = torch.empty(xs.lib().modit_workspace_bytes(dl.n, len(atm.p_bar), 16, nf, prec), dtype=torch.uint8,
                             device=dev)
            t, r = timed(lambda: xs.modit_compute(dl, nu_min, nu_max, N, T, P, n_gamma=16, n_fft=nf, prec=prec,
                                                  workspace=ws))
            ms += t
            sig.append(r.double())
            del ws
        out[name] = (ms, sig)
    res["fp64_ms"], res["fp32_ms"] = out["fp64"][0], out["fp32"][0]
    ms = 0.0
    lpf = []
    for dl in lines:
        t, r = timed(lambda: xs.xs_compute(dl, nu, T, P, prec=xs.PREC_MIXED))
        ms += t
        lpf.append(r.double())
    res["lpf_mixed_ms"] = ms
    d = []
    for m, l in zip(out["fp64"][1], lpf):
        mask = l > 1e-3 * l.max(dim=1, keepdim=True).values
        d.append(((m - l).abs() / l)[mask])
    d = torch.cat(d)
    res["vs_lpf_rel_diff"] = {"median": float(d.median()), "p99": float(d.sort().values[int(0.99 * (d.numel() - 1))]),
                              "where": "sigma_LPF > 1e-3 of the layer maximum; LPF cut at 25 cm^-1, MODIT uncut"}
    theta = W.theta_points(64)[0]
    for name, prec in (("fp64", xs.PREC_FP64), ("fp32", xs.PREC_MIXED)):
        mm = xs.EmissionModel(atm, prec=prec, device=dev, lines=lines, method="modit", n_gamma=16)
        F = mm.forward(W.THETA_STAR).clone()
        mm.set_observation(F * (1.0 + 0.01 * torch.as_tensor(W.std_normal(N), device=dev)), 0.01 * F)
        t, _ = timed(lambda: mm.logl_grad_async(theta))
        res[f"step_fwd_grad_{name}_ms"] = t
        del mm
        torch.cuda.empty_cache()
    d32 = torch.cat([((a - b).abs() / b.abs().amax(dim=1, keepdim=True)).flatten()
                     for a, b in zip(out["fp32"][1], out["fp64"][1])])
    res["fp32_vs_fp64_max_rel_to_layer_max"] = float(d32.max())
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale", choices=["scale", "emission"],
                    help="headline workload: the 10.2M-line precision form at scale (default) or the emission case")
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--layers", type=int, default=100,
                    help="layer count of the headline workload (100; fewer only for small profiling cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-errors", action="store_true", help="skip the mixed-vs-FP64 error block")
    ap.add_argument("--no-extra", action="store_true", help="skip the emission-workload line")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-modit", action="store_true", help="skip the MODIT measurement")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2105_14782_gb300 import _build
    if local == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    from paper_2105_14782_gb300 import xs

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    prec = xs.PREC_MIXED if args.prec == "mixed" else xs.PREC_FP64
    atm = atmosphere(args.workload, args.layers)
    e2e_steps = max(1, min(2, args.steps))
    res = step_bench(dev, stream, atm, prec, args.steps, args.warmup, rank, world, dist, e2e_steps)
    t_max = res["t_max"]
    roof = roofline(res, atm, args.workload, args.steps, n_sm, res["clocks"])
    fwd_ms, fwd_n, adj_ms, adj_n = res["prof"]
    skipped = []

    errors, fp64 = None, None
    if rank == 0 and not args.no_errors and prec == xs.PREC_MIXED:
        if elapsed() < WALL_BUDGET_S - 300:
            errors, fp64 = error_block(dev, atm, res["model"], res["theta"], stream)
        else:
            skipped.append("errors")
    del res["model"]
    torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(atm)

    extra = None
    if rank == 0 and world == 1 and not args.no_extra and args.workload == "scale":
        if elapsed() < WALL_BUDGET_S - 200:
            em = atmosphere("emission")
            r2 = step_bench(dev, stream, em, prec, 20, 3, rank, 1, None, 4)
            rf2 = roofline(r2, em, "emission", 20, n_sm, r2["clocks"])
            extra = {"emission": {"workload": WORKLOAD_TEXT["emission"], "value": r2["value"], "unit": "evals/s",
                                  "ms_per_step": r2["t_max"] / 20, "steps": 20, "warmup": 3,
                                  "evals_per_step": r2["evals_per_step"], "e2e": r2["e2e"], "roofline": rf2,
                                  "clocks": r2["clocks"], "gpu_launches": r2["launches"]}}
            del r2
            torch.cuda.empty_cache()
        else:
            skipped.append("extra")

    modit = None
    if rank == 0 and world == 1 and not args.no_modit:
        if elapsed() < WALL_BUDGET_S - 200:
            modit = {"emission": modit_stats(dev, atmosphere("emission"))}
            torch.cuda.empty_cache()
        else:
            skipped.append("modit")

    serve_stats = None
    if rank == 0 and world == 1 and not args.no_serve:
        if elapsed() < WALL_BUDGET_S - 120:
            serve_stats = serving(dev, WALL_BUDGET_S)
        else:
            skipped.append("serving")

    if rank == 0:
        L, N = len(atm.p_bar), len(atm.nu)
        line = {"metric": "Voigt line x grid x layer evals/s", "value": res["value"], "unit": "evals/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if prec == xs.PREC_MIXED else "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD_TEXT[args.workload] if L == 100 else
                           WORKLOAD_TEXT[args.workload].replace("100 layers", f"{L} layers"),
                           "step": "forward + gradient (logL and dlogL/dtheta, theta = T0, alpha, 2 log10 VMR, "
                                   "broadening scale)",
                           "precision": "FP32 Voigt + compensated FP32 sums, FP64 offsets/strengths, FP64 RT"
                           if prec == xs.PREC_MIXED else "FP64 throughout",
                           "evals_per_step": res["evals_per_step"], "in_cut_triples": res["triples"],
                           "l2": "inputs larger than L2: the per-step line records (tens of GB) are rewritten "
                                 "every step",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": res["e2e"], "clocks": res["clocks"],
                "gpu_launches": res["launches"],
                "kernel_ms_per_step": {"linesum_fwd": fwd_ms / args.steps, "linesum_adj": adj_ms / args.steps},
                "errors": errors, "fp64_path": fp64, "extra": extra, "serving": serve_stats, "modit": modit,
                "skipped": skipped, "wall_s": elapsed()}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
