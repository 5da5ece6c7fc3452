"""p-p calibration over a campaign of injections (Sec. 5.1, App. B) with the
GPU sampler: 32 signals drawn from the 4 s workload's prior (no SNR cut, so
the credible levels of the true values are uniform for a calibrated
sampler), each with its own noise; per parameter a KS test of the levels
against U(0, 1), combined by Fisher's method.  The error against the FP64
oracle is checked on a sampled subset of every injection's dead points (the
highest-weight one and one from the middle of the run)."""
import numpy as np
import pytest

import parity
import swig_inputs as si
from oracle import events, physics, pp
from oracle import likelihood as L

pytestmark = pytest.mark.gpu

swig = pytest.importorskip("paper_2607_28265_gb300.swig")

N_INJ = 32


def test_pp_calibration_campaign():
    base = si.config1()
    sampled = base.sampled()
    rng = np.random.default_rng(6000)
    levels = {s: [] for s in sampled}
    got, want = [], []
    for i in range(N_INJ):
        wl = si.config1()
        th = physics.prior_transform(rng.random(len(sampled)), wl.params)[0]
        wl.injection = th
        wl.target_snr = 0.0          # keep the prior draw (no rescaling)
        wl.noise_seed = 7000 + i
        ev, th_used = events.build_event(wl)
        ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
        ctx.set_sampler(nlive=200, nrep=20, steps_per_dim=5, seed=8000 + i, precision=swig.PREC_MIXED)
        r = ctx.run()
        thd, ll, lw = ctx.get_samples()
        assert r.status == 0
        for s in sampled:
            levels[s].append(pp.credible_level(thd[:, s], lw, th_used[s]))
        for j in (int(np.argmax(lw)), len(ll) // 2):
            got.append(ll[j])
            want.append(L.loglike(ev, thd[j]))
        ctx.close()
    parity.check("p-p campaign dead points (4 s H1, mixed, 32 injections)", np.array(got), np.array(want), 1e-6, 1e-6)
    pvals = [pp.ks_uniform_pvalue(levels[s]) for s in sampled]
    assert min(pvals) > 1e-3, dict(zip([si.PARAM_NAMES[s] for s in sampled], pvals))
    assert pp.fisher_combined(pvals) > 1e-3, pvals
