"""Benchmark: nested-sampling posteriors through the C-ABI library.

One step is one complete posterior: a Slice-within-Gibbs nested-sampling run
(Sec. 2.2, 2.3, 3.2 of the paper) from prior draws to the termination rule.
The metric is logL evaluations per second (all likelihood evaluations,
including the projection-only updates of cached blocks, as the paper counts
them) and wall-seconds per posterior (= ms_per_step / 1000).

``--workload`` picks the configuration (default ``cfg2``, the headline):

  cfg2      128 s H1/L1/V1 BNS, 259,585 bins/det, full grid, plain SwiG, mixed
  cfg5      cfg2 with the learned slice proposal (learned + mixed)
  cfg2-het  cfg2 with the heterodyned likelihood, 5,000 bins (Sec. 3.4)
  cfg2-het-tm  cfg2-het with t_c marginalised on 2,000 grid nodes over its
            prior and d_L sampled (Sec. 3.1, App. A; the paper's
            recommended configuration)
  cfg2-nss  cfg2 without Gibbs blocks (all sampled parameters in one block)
  cfg2-m3   cfg2 with M = 3 Gibbs sweeps per replacement (the paper's High-Res)
  cfg4      one batch of the injection campaign: four 3-detector events of
            32/64/128/256 s in one persistent launch (swig_run_batch)
  cfg1      4 s single detector, 4,017 bins, FP64, nlive 100
  cfg3      cfg1 data, heterodyned likelihood, 450 geometric bins, nlive 1000

Output: one JSON line on rank 0 (with ``sampler_profile``, the sampler's
device phase timers averaged over the timed posteriors).  ``--impl reference`` times the FP64 CPU
oracle on the same workload instead (bounded samples of likelihood
evaluations per step on the host cores).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import swig_inputs as si  # noqa: E402

SFU_OPS_PER_CLK_SM = 16   # sin/cos results per clock per SM (sm_100-class SFU), used if the probe fails
SFU_OPS_PER_BIN_DET = 2   # one sine and one cosine per bin and detector
# DRAM bytes (read + write) per logL evaluation inside k_ns_flow (512
# threads), from one ncu capture of a 2-iteration launch of the 128 s workload
# (10.03 MB + 0.31 MB over 107,944 evaluations; profiles/
# k_ns_flow_cfg2_hlv_128s_2iter.md), scaled to a full launch by its evaluations.
TRAFFIC_B_PER_EVAL = (10.032128e6 + 0.309504e6) / 107944
METRIC = "logL evals/s (128 s 3-det BNS) and wall-s/posterior, plain vs learned+mixed"

# workload name -> (event, sampler options, description)
WORKLOADS = {
    "cfg2": dict(event="cfg2", precision="mixed", likelihood="full", proposal="cov",
                 text="plain SwiG (covariance directions), full grid, mixed precision"),
    "cfg5": dict(event="cfg2", precision="mixed", likelihood="full", proposal="learned", learn_mix=1.0,
                 learn_interval=32, learn_steps=30,
                 text="learned slice proposal (MLP 13-256-256-26, BF16/FP32, every slice direction, retrained every "
                      "32 iterations with 30 Adam steps), full grid, mixed"),
    "cfg2-het": dict(event="cfg2", precision="mixed", likelihood="het", proposal="cov", het_bins=5000,
                     het_spacing=0, text="plain SwiG, heterodyned likelihood, 5000 bins of equal phase change"),
    "cfg2-het-tm": dict(event="cfg2", precision="mixed", likelihood="het", proposal="cov", het_bins=5000,
                        het_spacing=0, tmarg_nodes=2000,
                        text="plain SwiG, heterodyned likelihood (5000 bins of equal phase change), t_c "
                             "marginalised on 2000 nodes over its +-0.1 s prior, d_L sampled"),
    "cfg2-nss": dict(event="cfg2", precision="mixed", likelihood="full", proposal="cov", single_block=True,
                     text="unblocked nested slice sampling (one block of all sampled parameters), full grid, mixed"),
    "cfg2-m3": dict(event="cfg2", precision="mixed", likelihood="full", proposal="cov", sweeps=3,
                    text="plain SwiG, M = 3 Gibbs sweeps per replacement, full grid, mixed"),
    "cfg4": dict(event="campaign", precision="mixed", likelihood="full", proposal="cov",
                 text="campaign batch: 4 events (32/64/128/256 s, injections drawn from the prior, SNR 25) "
                      "in one persistent launch, plain SwiG, full grid, mixed"),
    "cfg1": dict(event="cfg1", precision="fp64", likelihood="full", proposal="cov", nlive=100,
                 text="plain SwiG, full grid, FP64"),
    "cfg3": dict(event="cfg1", precision="mixed", likelihood="het", proposal="cov", nlive=1000, het_bins=450,
                 het_spacing=1, text="plain SwiG, heterodyned likelihood, 450 geometric bins"),
}


CAMPAIGN_SECONDS = (32, 64, 128, 256)


def campaign_workloads(rank=0):
    """The four events of one campaign batch: 3-detector BNS injections drawn
    from the prior (seeds 1000 + i), segments of 32/64/128/256 s."""
    import dataclasses
    out = []
    for i, T in enumerate(CAMPAIGN_SECONDS):
        wl = si.config2(seed_index=10 + i + 100 * rank)
        out.append(dataclasses.replace(wl, df=1.0 / T, name=f"campaign_{T}s"))
    return out


def make_workload(name):
    spec = WORKLOADS[name]
    if spec["event"] == "campaign":
        return campaign_workloads()[2], spec
    wl = si.config2() if spec["event"] == "cfg2" else si.config1(nlive=spec.get("nlive", 100))
    if spec.get("single_block"):
        for p in wl.params:
            if p.mode == si.MODE_SAMPLE:
                p.block = 0
    wl.sweeps = spec.get("sweeps", 1)
    return wl, spec


def tmarg_params(wl):
    """The workload's prior with t_c marginalised over the same uniform range."""
    params = list(wl.params)
    p = params[si.IDX["tc"]]
    params[si.IDX["tc"]] = si.Param(si.PRIOR_UNIFORM, p.lo, p.hi, si.MODE_MARG)
    return params


def workload_description(wl, spec):
    dets = "/".join(wl.detectors)
    return (f"{wl.name}: {1.0 / wl.df:g} s, {dets}, {wl.f_min:g}-{wl.f_max:g} Hz, {wl.n_bins} bins/det, "
            f"{len(wl.sampled())} sampled params, nlive={wl.nlive}, nrep={wl.nrep}, "
            f"{wl.steps_per_dim} slice steps/dim, M={wl.sweeps}; {spec['text']}")


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def measure_sfu_peak():
    """The SFU roofline denominator measured on this GPU: compile and run
    paper_2607_28265_gb300/csrc/peak_probe.cu (__sincosf throughput, best of 5
    launches).  Returns (Top/s at the measured rate, source text); falls back
    to the unit-count derivation if the probe cannot run."""
    src = os.path.join(ROOT, "paper_2607_28265_gb300", "csrc", "peak_probe.cu")
    exe = os.path.join(ROOT, "_build", "peak_probe")
    try:
        os.makedirs(os.path.dirname(exe), exist_ok=True)
        nvcc = os.environ.get("NVCC", "nvcc")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True,
                       capture_output=True, timeout=300)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
        rows = [json.loads(l) for l in out.splitlines() if l.strip().startswith("{")]
        sfu = next(r for r in rows if r["kind"] == "sfu_sincos_results")
        return sfu["ops_per_s"] / 1e12, (f"measured on this GPU: {sfu['per_clk_per_sm_at_max_clock']:.2f} sin/cos "
                                        f"results per clk per SM at the {sfu['max_clock_khz'] / 1e3:.0f} MHz maximum "
                                        f"clock (peak_probe.cu, __sincosf, 64 warps/SM, best of 5)")
    except Exception as e:  # noqa: BLE001 - any failure falls back to the derived figure
        return (SFU_OPS_PER_CLK_SM * 152 * 2070.0e6 / 1e12,
                f"16 sin/cos per clk per SM x 152 SMs x 2070 MHz (derived; the probe failed: {type(e).__name__})")

def reduce_over_ranks(local, world, device="cuda"):
    """Elementwise max and sum over the ranks of a vector of per-rank figures
    (the caller takes times from the max and counts from the sum); a plain
    copy at world 1.  NCCL on the GPU arm, any backend whose tensors live on
    `device` (gloo on "cpu" in the tests)."""
    t = np.asarray(local, dtype=np.float64)
    if world == 1:
        return t.copy(), t.copy()
    import torch
    import torch.distributed as dist
    x = torch.tensor(t, device=device)
    tmax, tsum = x.clone(), x.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return tmax.cpu().numpy(), tsum.cpu().numpy()

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_campaign(args, rank, world):
    """cfg4: each step is one batch of four posteriors in one persistent launch."""
    import torch

    from paper_2607_28265_gb300 import swig
    from paper_2607_28265_gb300.workloads import build_context

    torch.cuda.set_device(0 if world == 1 else int(os.environ.get("LOCAL_RANK", rank)))
    spec = WORKLOADS["cfg4"]
    wls = campaign_workloads(rank)
    stream = torch.cuda.current_stream()
    built = [build_context(wl) for wl in wls]
    ctxs = [b[0] for b in built]
    for ctx in ctxs:
        ctx.set_stream(stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = swig.run_batch(ctxs)
        e1.record(stream)
        torch.cuda.synchronize()
        return res, e0.elapsed_time(e1)

    for _ in range(args.warmup):
        step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = sum(c.profile()["kernel_launches"] for c in ctxs)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clocks:
        out = [step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    launches = int(sum(c.profile()["kernel_launches"] for c in ctxs) - launches0)
    total_ms = sum(ms for _, ms in out)
    evals = sum(r.n_evals for res, _ in out for r in res)
    full = sum(r.n_sweep_evals for res, _ in out for r in res)
    # end to end: data and PSDs from pinned host memory, the batch, the samples back
    pinned = [[torch.from_numpy(np.ascontiguousarray(d)).pin_memory() for d in b[1]] for b in built]
    pinned_psd = [[torch.from_numpy(np.ascontiguousarray(p)).pin_memory() for p in b[2]] for b in built]
    h2d0 = sum(c.profile()["h2d_bytes"] for c in ctxs)
    d2h0 = sum(c.profile()["d2h_bytes"] for c in ctxs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ctx, dd, pp in zip(ctxs, pinned, pinned_psd):
        for i in range(len(dd)):
            ctx.set_data(i, dd[i].numpy())
            ctx.set_psd(i, pp[i].numpy())
    res = swig.run_batch(ctxs)
    for ctx in ctxs:
        ctx.get_samples()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3
    e2e_evals = sum(r.n_sweep_evals for r in res)  # full-grid evaluations, as `value`
    h2d = sum(c.profile()["h2d_bytes"] for c in ctxs) - h2d0
    d2h = sum(c.profile()["d2h_bytes"] for c in ctxs) - d2h0
    tmax, tsum = reduce_over_ranks([total_ms, evals, e2e_ms, e2e_evals, full], world)
    total_ms_max, e2e_ms_max = float(tmax[0]), float(tmax[2])
    evals_all, e2e_all, full_all = float(tsum[1]), float(tsum[3]), float(tsum[4])
    if rank != 0:
        return None
    n_post = len(wls) * args.steps
    bindet = sum(r.n_sweep_evals * 3 * wl.n_bins for res, _ in out for r, wl in zip(res, wls))
    peak, peak_source = measure_sfu_peak()
    achieved = SFU_OPS_PER_BIN_DET * bindet / (total_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": full_all / (total_ms_max * 1e-3), "unit": "logL evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
        "wall_s_per_posterior": total_ms_max / n_post / 1e3,
        "all_evals_per_s": evals_all / (total_ms_max * 1e-3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "; ".join(f"{wl.name}: {wl.n_bins} bins/det" for wl in wls) + "; " + spec["text"],
                   "name": "cfg4", "posteriors_per_step": len(wls), "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}",
                   "posteriors": [{"logz": r.logz, "logz_err": r.logz_err, "n_iter": r.n_iter} for r in out[-1][0]]},
        "e2e": {"value": e2e_all / (e2e_ms_max * 1e-3), "unit": "logL evals/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms_max},
        "gpu_launches": launches,
        "roofline": {"kernel": "k_ns_multi (campaign persistent kernel)", "bound": "alu", "achieved": achieved,
                     "peak": peak, "unit": "SFU Top/s", "frac": achieved / peak, "traffic": None,
                     "work_per_launch": "2 SFU ops x bin-detector evaluations of the four events",
                     "timing": "CUDA events around each batch (the batch's persistent launches and host steps)",
                     "peak_source": peak_source},
        "clocks": clocks.summary(),
    }
    if args.cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline("cfg4", seconds=args.cpu_seconds,
                                            evals_per_posterior=evals / max(1, n_post))
    return line


def run_gpu(args, rank, world):
    if args.workload == "cfg4":
        return run_campaign(args, rank, world)
    import torch

    from paper_2607_28265_gb300 import swig
    from paper_2607_28265_gb300.workloads import build_context

    torch.cuda.set_device(0 if world == 1 else int(os.environ.get("LOCAL_RANK", rank)))
    wl, spec = make_workload(args.workload)
    prec = swig.PREC_FP64 if spec["precision"] == "fp64" else swig.PREC_MIXED
    ctx, data, psds, th_inj = build_context(wl, seed_offset=1000 * rank, precision=prec)
    het = spec["likelihood"] == "het"
    n_tm = spec.get("tmarg_nodes", 0)
    if n_tm:
        ctx.set_prior(tmarg_params(wl))  # the same event, t_c now marginalised
    ctx.set_sampler(nlive=wl.nlive, nrep=wl.nrep, sweeps=wl.sweeps, steps_per_dim=wl.steps_per_dim,
                    seed=wl.sampler_seed + 1000 * rank, precision=prec,
                    likelihood=swig.LIKE_HET if het else swig.LIKE_FULL,
                    proposal=swig.PROPOSAL_LEARNED if spec["proposal"] == "learned" else swig.PROPOSAL_COV,
                    het_bins=spec.get("het_bins", 0), het_spacing=spec.get("het_spacing", 0),
                    het_fiducial=th_inj if het else None, tmarg_nodes=n_tm, learn_mix=spec.get("learn_mix", 0.0),
                    learn_interval=spec.get("learn_interval", 0), learn_steps=spec.get("learn_steps", 0))
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    peak_sfu, peak_source = measure_sfu_peak() if rank == 0 else (None, None)

    def step_device():
        flush.zero_()  # evict L2 between steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = ctx.run()
        e1.record(stream)
        torch.cuda.synchronize()
        prof = ctx.profile()
        return r, e0.elapsed_time(e1), prof

    # warm-up (includes the one-off host preparation of the grid tables)
    for _ in range(args.warmup):
        step_device()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    results = []
    launches0 = ctx.profile()["kernel_launches"]
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clocks:
        for _ in range(args.steps):
            results.append(step_device())
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = int(ctx.profile()["kernel_launches"] - launches0)
    total_ms = sum(ms for _, ms, _ in results)
    total_evals = sum(r.n_evals for r, _, _ in results)
    full_evals = sum(r.n_sweep_evals for r, _, _ in results)
    pers_ms = sum(p["persistent_ms"] for _, _, p in results)
    pers_launch = sum(p["persistent_launches"] for _, _, p in results)
    bindet = sum(p["bin_det_evals"] for _, _, p in results)

    # end to end through the public API from pinned host buffers: set data and
    # PSDs (host -> device inside the library), run, read back the samples
    pinned = [torch.from_numpy(np.ascontiguousarray(d)).pin_memory() for d in data]
    pinned_psd = [torch.from_numpy(np.ascontiguousarray(s)).pin_memory() for s in psds]
    e2e_ms, e2e_evals, e2e_full = [], 0, 0
    h2d0, d2h0 = ctx.profile()["h2d_bytes"], ctx.profile()["d2h_bytes"]
    for _ in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(len(pinned)):
            ctx.set_data(i, pinned[i].numpy())
            ctx.set_psd(i, pinned_psd[i].numpy())
        r = ctx.run()
        th_s, ll_s, lw_s = ctx.get_samples()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_evals += r.n_evals
        e2e_full += r.n_sweep_evals
    n_e2e = max(1, args.e2e_steps)
    h2d = (ctx.profile()["h2d_bytes"] - h2d0) / n_e2e
    d2h = (ctx.profile()["d2h_bytes"] - d2h0) / n_e2e

    # the metric's comparison (cfg2): the learned proposal with mixed precision
    # on the same event, same K and W, then both arms' posteriors side by side
    arms = None
    if args.workload == "cfg2" and args.learned_arm:
        th_p, ll_p, lw_p = ctx.get_samples()
        ls = WORKLOADS["cfg5"]
        ctx.set_sampler(nlive=wl.nlive, nrep=wl.nrep, sweeps=wl.sweeps, steps_per_dim=wl.steps_per_dim,
                        seed=wl.sampler_seed + 1000 * rank, precision=prec, proposal=swig.PROPOSAL_LEARNED,
                        learn_mix=ls.get("learn_mix", 0.0), learn_interval=ls.get("learn_interval", 0),
                        learn_steps=ls.get("learn_steps", 0))
        for _ in range(args.warmup):
            step_device()
        learned = [step_device() for _ in range(args.steps)]
        th_l, ll_l, lw_l = ctx.get_samples()
        # the run-to-run variation of plain SwiG itself (another seed), the
        # scale against which the arms' difference is read
        ctx.set_sampler(nlive=wl.nlive, nrep=wl.nrep, sweeps=wl.sweeps, steps_per_dim=wl.steps_per_dim,
                        seed=wl.sampler_seed + 1000 * rank + 1, precision=prec)
        r_b, _, _ = step_device()
        th_b, ll_b, lw_b = ctx.get_samples()
        arms = {"plain": _arm_summary(results, "plain SwiG: covariance directions, mixed precision"),
                "learned": _arm_summary(learned, "learned + mixed: " + ls["text"]),
                "posterior_comparison": {
                    "plain_vs_learned": _compare_posteriors(wl, (th_p, lw_p), (th_l, lw_l), results[-1][0],
                                                            learned[-1][0]),
                    "plain_vs_plain_other_seed": _compare_posteriors(wl, (th_p, lw_p), (th_b, lw_b), results[-1][0],
                                                                     r_b)}}

    # max of the times and sum of the counts over ranks
    tmax, tsum = reduce_over_ranks([total_ms, total_evals, sum(e2e_ms), e2e_evals, full_evals, e2e_full], world)
    total_ms_max, e2e_ms_max = float(tmax[0]), float(tmax[2])
    evals_all, e2e_evals_all, full_all = float(tsum[1]), float(tsum[3]), float(tsum[4])
    e2e_full_all = float(tsum[5])
    if rank != 0:
        return None

    clk = clocks.summary()
    sm_mhz_max = 2070.0
    peak = peak_sfu  # SFU Top/s, measured on this GPU by peak_probe.cu
    achieved = SFU_OPS_PER_BIN_DET * bindet / (pers_ms * 1e-3) / 1e12 if pers_ms > 0 else 0.0
    n_bins_eval = spec.get("het_bins", 0) + 1 if het else wl.n_bins
    kernel = "k_ns_het (persistent SwiG kernel, heterodyned)" if het else "k_ns_flow (persistent SwiG kernel, dataflow)"
    traffic = (TRAFFIC_B_PER_EVAL * total_evals / max(1, pers_launch)
               if TRAFFIC_B_PER_EVAL is not None and args.workload == "cfg2" else None)
    line = {
        "metric": METRIC,
        # full-grid (or heterodyned) evaluations: those that run the sweep, the
        # same kind the CPU oracle arm times; all evaluations (projection-only
        # updates from the cached sums included) in all_evals_per_s
        "value": full_all / (total_ms_max * 1e-3),
        "unit": "logL evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps,
        "wall_s_per_posterior": total_ms_max / args.steps / 1e3,
        "all_evals_per_s": evals_all / (total_ms_max * 1e-3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if spec["precision"] == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": workload_description(wl, spec), "name": args.workload,
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}",
                   "posterior": {"logz": results[-1][0].logz, "logz_err": results[-1][0].logz_err,
                                 "ess": results[-1][0].ess, "n_iter": results[-1][0].n_iter,
                                 "n_dead": results[-1][0].n_dead}},
        "e2e": {"value": e2e_full_all / (e2e_ms_max * 1e-3), "unit": "logL evals/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": e2e_ms_max / n_e2e},
        "gpu_launches": launches,
        "roofline": {
            "kernel": kernel,
            "bound": "alu",
            "achieved": achieved,
            "peak": peak,
            "unit": "SFU Top/s",
            "frac": achieved / peak if peak else None,
            "traffic": traffic,
            "traffic_unit": "bytes per launch (ncu, 2-iteration capture scaled by evaluations)",
            "work_per_launch": (f"2 SFU ops x bin-detector evaluations (full evaluations x {len(wl.detectors)} x "
                                f"{n_bins_eval} {'bin edges' if het else 'bins'})"),
            "launches": int(pers_launch),
            "avg_launch_ms": pers_ms / max(1, pers_launch),
            "peak_source": peak_source,
        },
        "clocks": clk,
    }
    if n_tm:
        line["roofline"]["kernel"] = ("k_ns_het (persistent SwiG kernel, heterodyned, t_c marginalised: bin pass "
                                      "plus the non-uniform FFT time pass)")
    if args.cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload, seconds=args.cpu_seconds,
                                            evals_per_posterior=total_evals / max(1, args.steps))
    # the sampler's own device counters, averaged over the timed posteriors:
    # phase times, chain 0's control cycles by part, sweep-unit cycles
    prof_keys = ("rounds", "boundary_s", "control_s", "wait_control_s", "sweep_s", "wait_sweep_s", "cyc_result",
                 "cyc_step", "cyc_prop", "cyc_free", "cyc_setup", "n_free", "n_setup", "n_step", "f_units",
                 "f_unit_cyc", "f_idle_cyc")
    line["sampler_profile"] = {k: float(np.mean([p.get(k, 0.0) for _, _, p in results])) for k in prof_keys}
    if arms is not None:
        line["arms"] = arms
    if prof_learn := sum(p.get("learn_ms", 0.0) for _, _, p in results):
        line["learned"] = {"train_ms_per_posterior": prof_learn / args.steps,
                           "retrainings_per_posterior": sum(p.get("learn_rounds", 0) for _, _, p in results) / args.steps}
    return line


def _arm_summary(results, text):
    """Wall-s per posterior and the posteriors' figures of one arm's timed steps."""
    ms = [m for _, m, _ in results]
    return {"text": text, "wall_s_per_posterior": float(np.mean(ms)) / 1e3,
            "wall_s_each": [m / 1e3 for m in ms],
            "logz": [r.logz for r, _, _ in results], "logz_err": [r.logz_err for r, _, _ in results],
            "ess": [r.ess for r, _, _ in results], "n_evals": [r.n_evals for r, _, _ in results],
            "n_full_evals": [r.n_sweep_evals for r, _, _ in results],
            "train_ms": [p.get("learn_ms", 0.0) for _, _, p in results],
            "retrainings": [p.get("learn_rounds", 0.0) for _, _, p in results]}


def _compare_posteriors(wl, a, b, ra, rb):
    """Evidence difference and per-parameter weighted two-sample KS (Kish
    effective sizes) between two runs' weighted samples (theta, log w)."""
    out = {"dlogz": rb.logz - ra.logz, "dlogz_err": math.hypot(ra.logz_err, rb.logz_err), "ks": {}}
    wa, wb = np.exp(a[1] - a[1].max()), np.exp(b[1] - b[1].max())
    for slot in wl.sampled():
        d, p = _weighted_ks(a[0][:, slot], wa, b[0][:, slot], wb)
        out["ks"][si.PARAM_NAMES[slot]] = {"D": d, "p": p}
    return out


def _weighted_ks(x1, w1, x2, w2):
    """Two-sample Kolmogorov-Smirnov distance of weighted samples and its
    asymptotic p-value with n = n1 n2 / (n1 + n2) from the Kish effective sizes."""
    from scipy import stats
    w1, w2 = w1 / np.sum(w1), w2 / np.sum(w2)
    grid = np.sort(np.concatenate([x1, x2]))
    o1, o2 = np.argsort(x1), np.argsort(x2)
    c1 = np.concatenate([[0.0], np.cumsum(w1[o1])])
    c2 = np.concatenate([[0.0], np.cumsum(w2[o2])])
    d = float(np.max(np.abs(c1[np.searchsorted(x1[o1], grid, side="right")] -
                            c2[np.searchsorted(x2[o2], grid, side="right")])))
    n1, n2 = 1.0 / np.sum(w1 ** 2), 1.0 / np.sum(w2 ** 2)
    return d, float(stats.kstwobign.sf(d * math.sqrt(n1 * n2 / (n1 + n2))))


# ---------------------------------------------------------------------------
# CPU oracle (the baseline leg and the reference arm)
# ---------------------------------------------------------------------------
_EV = None


def _worker_init(name):
    """Hold the workload's synthetic event (and heterodyne tables) in the oracle."""
    global _EV
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import events
    from oracle import likelihood as L
    wl, spec = make_workload(name)
    ev, th = events.build_event(wl)
    if spec.get("tmarg_nodes"):
        ev = L.Event(ev.freqs, ev.df, ev.data, ev.psds, ev.detectors, ev.gmst, tmarg_params(wl))
        wl.params = ev.params
    het = L.het_setup(ev, th, spec["het_bins"], spacing="phase" if spec.get("het_spacing", 0) == 0 else "geometric") \
        if spec["likelihood"] == "het" else None
    _EV = (wl, ev, het, spec.get("tmarg_nodes", 0))


def _worker_evals(args):
    seed, n = args
    from oracle import likelihood as L
    from oracle import physics
    wl, ev, het, n_tm = _EV
    rng = np.random.default_rng(seed)
    ns = len(wl.sampled())
    t0 = time.perf_counter()
    for _ in range(n):
        t = physics.prior_transform(rng.random(ns), wl.params)[0]
        if het is None:
            L.loglike(ev, t)
        elif n_tm:
            L.het_loglike_time_marg(ev, het, t, n_tm)
        else:
            L.het_loglike(ev, het, t)
    return n, time.perf_counter() - t0


class OraclePool:
    """The FP64 oracle's logL on all host cores (spawned worker processes,
    each holding the synthetic event)."""

    def __init__(self, name):
        import multiprocessing as mp
        self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_worker_init, initargs=(name,))
        n0, t0 = self.pool.apply(_worker_evals, ((12345, 2),))
        self.per_eval = t0 / max(1, n0)
        self.seed = 100

    def sample(self, seconds):
        n_each = max(1, int(seconds / self.per_eval))
        t_start = time.perf_counter()
        res = self.pool.map(_worker_evals, [(self.seed + i, n_each) for i in range(self.cores)])
        wall = time.perf_counter() - t_start
        self.seed += self.cores
        total = sum(r[0] for r in res)
        return total, wall

    def close(self):
        self.pool.close()
        self.pool.join()


def _sample_text(name, total, cores, extra):
    wl, spec = make_workload(name)
    what = (f"heterodyned logL ({spec['het_bins']} bins)" if spec["likelihood"] == "het"
            else f"logL on the full {len(wl.detectors)} x {wl.n_bins}-bin grid")
    if spec.get("tmarg_nodes"):
        what += f" with t_c marginalised on {spec['tmarg_nodes']} nodes"
    return f"{total} FP64 oracle evaluations of {what} at prior draws, {cores} spawned processes, {extra}"


def cpu_baseline(name, seconds=15.0, evals_per_posterior=None):
    """Oracle logL evaluations/s over all host cores, on a bounded sample."""
    pool = OraclePool(name)
    try:
        total, wall = pool.sample(seconds)
    finally:
        pool.close()
    rate = total / wall
    out = {"value": rate, "unit": "logL evals/s", "cores": pool.cores, "kind": "oracle",
           "sample": _sample_text(name, total, pool.cores, f"{wall:.1f} s")}
    if evals_per_posterior:
        out["wall_s_per_posterior_extrapolated"] = evals_per_posterior / rate
    return out


def run_reference(args, rank, world):
    """The oracle arm: each step is a bounded sample of logL evaluations of
    the same workload on all host cores; value = evaluations/s."""
    if rank != 0:
        return None
    wl, spec = make_workload(args.workload)
    pool = OraclePool(args.workload)
    per_step_s = max(2.0, args.cpu_seconds / 2)
    try:
        for _ in range(args.warmup):
            pool.sample(1.0)
        total, t_all = 0, 0.0
        for _ in range(args.steps):
            n, w = pool.sample(per_step_s)
            total += n
            t_all += w
    finally:
        pool.close()
    value = total / t_all
    sample = _sample_text(args.workload, total, pool.cores, f"over {args.steps} steps")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "logL evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_all / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_description(wl, spec), "name": args.workload,
                   "note": "FP64 CPU oracle of the same method, bounded samples per step"},
        "cpu_baseline": {"value": value, "unit": "logL evals/s", "cores": pool.cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "logL evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--impl", choices=["swig", "reference"], default="swig")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cfg2")
    ap.add_argument("--no-learned-arm", dest="learned_arm", action="store_false",
                    help="cfg2 only: skip the learned-proposal arm of the metric's comparison")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "swig":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    line = run_reference(args, rank, world) if args.impl == "reference" else run_gpu(args, rank, world)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl == "swig":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
