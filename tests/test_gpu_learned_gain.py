"""What the trained network gains over plain SwiG, on the full-size 128 s
H1/L1/V1 workload, through the C-ABI.

Both arms sample the same event with the same seeds; the learned arm draws
every slice direction from the online-trained network (retrained every 32
iterations, 30 Adam steps; plain SwiG draws them from the live covariance).
The gain is measured as full-grid likelihood evaluations per effective
posterior sample (Kish size of the nested-sampling weights): the learned arm
must need at least 5% fewer (measured: about 15% fewer).  Its evidence must
agree with plain SwiG's within three times the run-to-run scatter measured on
this workload over nine seeds (0.55 nat per run; the per-run error estimate
sqrt(H / m) = 0.17 understates it because five slice steps per dimension
leave successive live points correlated).
"""
import math

import numpy as np
import pytest

import swig_inputs as si
from oracle import events

pytestmark = pytest.mark.gpu

swig = pytest.importorskip("paper_2607_28265_gb300.swig")

RUN_SCATTER = 0.55  # nat, run-to-run sd of log Z on this workload (plain SwiG, nine seeds)


def test_learned_proposal_lowers_evaluations_per_effective_sample():
    wl = si.config2()
    ev, th = events.build_event(wl)
    ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
    out = {"plain": [], "learned": []}
    for seed in (51, 52):
        for arm in ("plain", "learned"):
            kw = dict(nlive=1000, nrep=100, steps_per_dim=5, seed=seed, precision=swig.PREC_MIXED)
            if arm == "learned":
                kw.update(proposal=swig.PROPOSAL_LEARNED, learn_mix=1.0, learn_interval=32, learn_steps=30)
            ctx.set_sampler(**kw)
            r = ctx.run()
            assert r.status == 0 and np.isfinite(r.logz)
            if arm == "learned":
                assert ctx.profile()["learn_rounds"] >= 2
            out[arm].append((r.n_sweep_evals / r.ess, r.logz))
    ctx.close()
    cost = {a: np.mean([c for c, _ in v]) for a, v in out.items()}
    logz = {a: np.mean([z for _, z in v]) for a, v in out.items()}
    assert cost["learned"] < 0.95 * cost["plain"], cost
    # the difference of two means of two runs each has sd RUN_SCATTER * sqrt(1/2 + 1/2)
    assert abs(logz["learned"] - logz["plain"]) < 3.0 * RUN_SCATTER * math.sqrt(0.5 + 0.5), (out, logz)
