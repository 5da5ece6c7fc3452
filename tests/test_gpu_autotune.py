"""Launch-shape autotuning of the full-grid persistent sampler
(swig_autotune), through the C-ABI.

The tuner runs a few NS iterations with each launch shape (slice parts per
sweep request, one- or two-ended stepping-out) and keeps the fastest.  Here:
it reports four candidates with positive rates and keeps the fastest; the
kept shape, set explicitly, reproduces the tuned run bit for bit; the tuned
run's dead points equal the oracle's logL; settings without a launch shape
(FP64) report no candidates and change nothing.
"""
import numpy as np
import pytest

import parity
import swig_inputs as si
from oracle import events
from oracle import likelihood as L

pytestmark = pytest.mark.gpu

swig = pytest.importorskip("paper_2607_28265_gb300.swig")


def test_autotune_keeps_the_fastest_shape_and_valid_results():
    wl = si.config1()
    ev, th = events.build_event(wl)
    ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
    kw = dict(nlive=200, nrep=20, steps_per_dim=5, seed=17, precision=swig.PREC_MIXED)
    ctx.set_sampler(**kw)
    cands, chosen = ctx.autotune(iters=6)
    assert len(cands) == 4 and all(rate > 0 for _, _, rate in cands), cands
    assert {(g, o) for g, o, _ in cands} == {(1, 0), (1, 1), (2, 0), (3, 0)}
    assert chosen == max(cands, key=lambda t: t[2])[:2]
    r1 = ctx.run()
    thd, ll, lw = ctx.get_samples()
    assert r1.status == 0
    ctx.set_sampler(**kw, flow_parts=chosen[0], stepout_one_end=chosen[1])
    r2 = ctx.run()
    assert r2.logz == r1.logz and r2.n_evals == r1.n_evals
    rng = np.random.default_rng(3)
    idx = rng.choice(len(ll), 8, replace=False)
    want = np.array([L.loglike(ev, thd[i]) for i in idx])
    parity.check("autotuned sampler dead points (4 s H1, mixed)", ll[idx], want, 1e-6, 1e-6)
    # FP64: no launch shape
    ctx.set_sampler(nlive=200, nrep=20, steps_per_dim=5, seed=17, precision=swig.PREC_FP64)
    cands, chosen = ctx.autotune(iters=2)
    assert cands == [] and chosen is None
    ctx.close()


def test_autotune_argument_errors():
    wl = si.config1()
    ev, th = events.build_event(wl)
    ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
    ctx.set_sampler(nlive=200, nrep=20, precision=swig.PREC_MIXED)
    with pytest.raises(swig.SwigError):
        ctx.autotune(iters=0)
    with pytest.raises(swig.SwigError):
        ctx.set_sampler(nlive=200, nrep=20, precision=swig.PREC_MIXED, flow_parts=5)
    ctx.close()
