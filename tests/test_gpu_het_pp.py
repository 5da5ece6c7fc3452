"""p-p calibration of the heterodyned likelihood (Sec. 3.4, Sec. 5.1, App. A)
on a three-detector workload, with t_c sampled and with t_c marginalised.

The paper finds sampled t_c under-covered under relative binning and
calibration restored by marginalising it.  Here: H1/L1/V1, 8 s at 20-1024 Hz,
signals drawn from the prior (Mc U[1.1, 1.3], q U[0.5, 1], d_L U[20, 120]
Mpc, t_c U[-0.03, 0.03] s, the +-0.03 s window of the paper's time-marginalised
analysis), each with its own noise; 2,500 phase-spaced bins with the fiducial
at the injection; nlive 200, k 20, {Mc, q, t_c} one block.  Marginalised: 4,096
nodes over the window (15 us apart, below the t_c posterior width), t_c
reconstructed from the node weights.  Per parameter a KS test of the credible
levels of the true values against U(0, 1), combined by Fisher's method.  The
number of injections per mode is SWIG_HET_PP_INJECTIONS (default 32).
"""
import math
import os

import numpy as np
import pytest

import parity
import swig_inputs as si
from oracle import events, physics, pp

pytestmark = pytest.mark.gpu

swig = pytest.importorskip("paper_2607_28265_gb300.swig")

N_INJ = int(os.environ.get("SWIG_HET_PP_INJECTIONS", "32"))
TC_HALF = 0.03
N_BINS = 2500
N_NODES = 4096


def _params(tc_mode):
    P = si.Param
    fixed = si.MODE_FIXED
    return [P(si.PRIOR_UNIFORM, 1.1, 1.3, block=0), P(si.PRIOR_UNIFORM, 0.5, 1.0, block=0),
            P(si.PRIOR_UNIFORM, 0, 0, fixed, 0.0), P(si.PRIOR_UNIFORM, 0, 0, fixed, 0.0),
            P(si.PRIOR_UNIFORM, 0, 0, fixed, 0.0), P(si.PRIOR_UNIFORM, 0, 0, fixed, 0.0),
            P(si.PRIOR_UNIFORM, 20.0, 120.0, block=1), P(si.PRIOR_UNIFORM, 0, 0, fixed, 0.4),
            P(si.PRIOR_UNIFORM, 0, 0, fixed, 0.3), P(si.PRIOR_UNIFORM, 0, 0, fixed, 1.2),
            P(si.PRIOR_UNIFORM, 0, 0, fixed, 0.5),
            P(si.PRIOR_UNIFORM, -TC_HALF, TC_HALF, tc_mode, block=0),
            P(si.PRIOR_UNIFORM, 0.0, 2 * math.pi, si.MODE_MARG, block=2)]


@pytest.mark.parametrize("mode", ["sampled", "marginalised"])
def test_heterodyned_pp(mode):
    base = _params(si.MODE_SAMPLE)
    sampled = [i for i, p in enumerate(base) if p.mode == si.MODE_SAMPLE]
    rng = np.random.default_rng(9100)
    levels = {s: [] for s in sampled}
    for i in range(N_INJ):
        th = physics.prior_transform(rng.random(len(sampled)), base)[0]
        wl = si.Workload(f"het_pp_{i}", 20.0, 1024.0, 0.125, ("H1", "L1", "V1"), base, th, 0.0,
                         noise_seed=9200 + i, sampler_seed=9300 + i, nlive=200, nrep=20, steps_per_dim=5)
        ev, th_used = events.build_event(wl)
        ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
        marg = mode == "marginalised"
        ctx.set_sampler(nlive=200, nrep=20, steps_per_dim=5, seed=9300 + i, precision=swig.PREC_MIXED,
                        likelihood=swig.LIKE_HET, het_bins=N_BINS, het_spacing=0, het_fiducial=th_used,
                        tmarg_nodes=N_NODES if marg else 0)
        ctx.set_prior(_params(si.MODE_MARG if marg else si.MODE_SAMPLE))
        r = ctx.run()
        assert r.status == 0
        thd, ll, lw = ctx.get_samples()
        for s in sampled:
            levels[s].append(pp.credible_level(thd[:, s], lw, th_used[s]))
        ctx.close()
    pvals = {si.PARAM_NAMES[s]: pp.ks_uniform_pvalue(levels[s]) for s in sampled}
    combined = pp.fisher_combined(list(pvals.values()))
    parity.note(f"heterodyned p-p, t_c {mode}", injections=N_INJ, ks_p=pvals, fisher_p=combined)
    assert min(pvals.values()) > 1e-3, pvals
    assert combined > 1e-3, (pvals, combined)
