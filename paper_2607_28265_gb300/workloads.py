"""Synthetic events through the library's own API, and small profiling cases.

``build_context(wl)`` loads a workload (grid, detectors, PSDs, prior) into a
context and makes its data with the library itself: the injection is mapped
from the unit cube by ``swig_prior_transform`` and its strain computed on the
device by ``swig_inject`` (FP64), plus the workload's seeded noise.

Run as a module it executes one small case for a profiler capture::

    python -m paper_2607_28265_gb300.workloads sampler --max-iter 2
    python -m paper_2607_28265_gb300.workloads loglike --batch 1000
    python -m paper_2607_28265_gb300.workloads het --batch 1000 --bins 1000
    python -m paper_2607_28265_gb300.workloads sampler-het --max-iter 2 --bins 5000
    python -m paper_2607_28265_gb300.workloads sampler-het --max-iter 2 --bins 5000 --tmarg-nodes 2000
    python -m paper_2607_28265_gb300.workloads learned --max-iter 2

``sampler``: the persistent nested-sampling kernel on the 128 s H1/L1/V1
workload for --max-iter outer iterations (one launch); ``loglike``: one batch
of the full-grid mixed-precision likelihood; ``het``: one batch of the
heterodyned likelihood; ``sampler-het``: the heterodyned persistent sampler
kernel (fiducial at the injection); ``learned``: the learned-proposal sampler
(its first training of the network, then the persistent kernel).
``--tmarg-nodes N`` marginalises t_c over
its prior on N grid nodes in the heterodyned cases.  Each case exits non-zero
on any library error.
"""
from __future__ import annotations

import argparse
import math

import numpy as np

import swig_inputs as si

from . import swig


def build_context(wl, seed_offset=0, precision=swig.PREC_MIXED):
    """Context with wl's grid, detectors, PSDs, prior and a synthetic event
    (library-computed injection + seeded noise).  Returns (ctx, data, psds,
    theta_injected)."""
    ctx = swig.Context(0)
    ctx.set_grid(wl.f_min, wl.f_max, wl.df)
    for i, name in enumerate(wl.detectors):
        ctx.set_detector(i, *si.site_vectors(name))
    ctx.set_time_ref(si.gmst_from_gps(si.REFERENCE_GPS))
    psds = wl.psds()
    for i, s in enumerate(psds):
        ctx.set_psd(i, s)
    ctx.set_prior(wl.params)
    if wl.inj_unit:
        u = np.asarray(wl.injection)
        sampled = wl.sampled()
        th = ctx.prior_transform(u[sampled][None, :])[0]
        th[si.IDX["phic"]] = 2.0 * math.pi * u[si.IDX["phic"]]
    else:
        th = np.asarray(wl.injection, dtype=np.float64).copy()
    noise = np.array(wl.noise())
    data, th_used = ctx.inject(th, len(wl.detectors), target_snr=wl.target_snr, noise=noise)
    for i in range(len(wl.detectors)):
        ctx.set_data(i, data[i])
    ctx.set_sampler(nlive=wl.nlive, nrep=wl.nrep, sweeps=wl.sweeps, steps_per_dim=wl.steps_per_dim,
                    seed=wl.sampler_seed + seed_offset, precision=precision)
    return ctx, data, psds, th_used


def _prior_draws(ctx, params, n, seed):
    rng = np.random.default_rng(seed)
    n_sampled = sum(1 for p in params if p.mode == si.MODE_SAMPLE)
    return ctx.prior_transform(rng.random((n, n_sampled)))


def main(argv=None):
    ap = argparse.ArgumentParser(description="small profiling cases on the 128 s three-detector workload")
    ap.add_argument("case", choices=["sampler", "sampler-het", "loglike", "het", "learned"])
    ap.add_argument("--max-iter", type=int, default=2)
    ap.add_argument("--batch", type=int, default=1000)
    ap.add_argument("--bins", type=int, default=1000)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--tmarg-nodes", type=int, default=0)
    a = ap.parse_args(argv)
    wl = si.config2()
    ctx, data, psds, th = build_context(wl)
    params = list(wl.params)
    if a.tmarg_nodes:
        p = params[si.IDX["tc"]]
        params[si.IDX["tc"]] = si.Param(si.PRIOR_UNIFORM, p.lo, p.hi, si.MODE_MARG)
        ctx.set_prior(params)
    if a.case == "sampler":
        ctx.set_sampler(nlive=wl.nlive, nrep=wl.nrep, sweeps=wl.sweeps, steps_per_dim=wl.steps_per_dim,
                        seed=wl.sampler_seed, precision=swig.PREC_MIXED, max_iter=a.max_iter)
        for _ in range(a.repeat):
            r = ctx.run()
        print(f"sampler: n_iter={r.n_iter} n_evals={r.n_evals} logz={r.logz:.3f}")
    elif a.case == "learned":
        ctx.set_sampler(nlive=wl.nlive, nrep=wl.nrep, sweeps=wl.sweeps, steps_per_dim=wl.steps_per_dim,
                        seed=wl.sampler_seed, precision=swig.PREC_MIXED, max_iter=a.max_iter,
                        proposal=swig.PROPOSAL_LEARNED, learn_mix=1.0, learn_interval=32, learn_steps=30)
        for _ in range(a.repeat):
            r = ctx.run()
        print(f"learned: n_iter={r.n_iter} n_evals={r.n_evals} logz={r.logz:.3f}")
    elif a.case == "sampler-het":
        ctx.set_sampler(nlive=wl.nlive, nrep=wl.nrep, sweeps=wl.sweeps, steps_per_dim=wl.steps_per_dim,
                        seed=wl.sampler_seed, likelihood=swig.LIKE_HET, het_bins=a.bins, het_fiducial=th,
                        max_iter=a.max_iter, tmarg_nodes=a.tmarg_nodes)
        for _ in range(a.repeat):
            r = ctx.run()
        print(f"sampler-het: n_iter={r.n_iter} n_evals={r.n_evals} logz={r.logz:.3f}")
    else:
        if a.case == "het":
            ctx.set_sampler(nlive=wl.nlive, nrep=wl.nrep, likelihood=swig.LIKE_HET, het_bins=a.bins,
                            het_fiducial=th, tmarg_nodes=a.tmarg_nodes)
        thetas = _prior_draws(ctx, params, a.batch, 7)
        for _ in range(a.repeat):
            out = ctx.loglike_batch(thetas)
        print(f"{a.case}: batch={a.batch} finite={int(np.isfinite(out).sum())} max={out.max():.3f}")
    ctx.close()


if __name__ == "__main__":
    main()
