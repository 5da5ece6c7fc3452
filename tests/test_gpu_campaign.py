"""Campaign runs (config 4) through swig_run_batch: events sharing one
persistent launch give exactly the results of separate runs (the 4 s and 8 s
events of the first test land in different launches: grids more than 1.5x
apart do not share one), and events that cannot share a launch run on their
own inside the same call."""
import dataclasses

import numpy as np
import pytest

import swig_inputs as si
from oracle import events

pytestmark = pytest.mark.gpu

swig = pytest.importorskip("paper_2607_28265_gb300.swig")


def _contexts(specs):
    out = []
    for wl, extra in specs:
        ev, th = events.build_event(wl)
        ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
        ctx.set_sampler(nlive=wl.nlive, nrep=wl.nrep, steps_per_dim=5, seed=wl.sampler_seed,
                        precision=swig.PREC_MIXED, **extra(th))
        out.append(ctx)
    return out


def _specs():
    base = si.config1(nlive=200)
    specs = []
    for i, df in enumerate((0.25, 0.125, 0.25)):
        wl = dataclasses.replace(base, df=df, noise_seed=9100 + i, sampler_seed=9200 + i, name=f"camp{i}")
        specs.append((wl, lambda th: {}))
    return specs


def _same(a, b):
    return a.logz == b.logz and a.n_dead == b.n_dead and a.n_evals == b.n_evals


def test_batch_equals_separate_runs():
    specs = _specs()
    single = []
    for ctx in _contexts(specs):
        r = ctx.run()
        single.append((r, ctx.get_samples()))
        ctx.close()
    ctxs = _contexts(specs)
    res = swig.run_batch(ctxs)
    for (r1, (t1, l1, w1)), r2, ctx in zip(single, res, ctxs):
        t2, l2, w2 = ctx.get_samples()
        assert _same(r1, r2), (r1, r2)
        assert np.array_equal(t1, t2) and np.array_equal(l1, l2) and np.array_equal(w1, w2)
        assert r2.status == 0
        ctx.close()


def test_batch_with_an_event_that_runs_alone():
    """A heterodyned event cannot share the full-grid launch; it runs alone
    and the others still share theirs."""
    specs = _specs()
    het_wl = dataclasses.replace(si.config1(nlive=200), noise_seed=9300, sampler_seed=9301, name="camphet")
    specs.insert(1, (het_wl, lambda th: {"likelihood": swig.LIKE_HET, "het_bins": 300, "het_fiducial": th}))
    single = []
    for ctx in _contexts(specs):
        single.append(ctx.run())
        ctx.close()
    ctxs = _contexts(specs)
    res = swig.run_batch(ctxs)
    for r1, r2 in zip(single, res):
        assert _same(r1, r2), (r1, r2)
    for ctx in ctxs:
        ctx.close()


def test_batch_three_detectors():
    """Three-detector 8 s events (phase marginalised, 12 parameters) sharing
    one launch equal separate runs."""
    specs = []
    for i, df in enumerate((1 / 8, 1 / 8)):
        wl = dataclasses.replace(si.config2(nlive=200, seed_index=5 + i), df=df, name=f"camp3d{i}")
        specs.append((wl, lambda th: {"max_iter": 40}))
    single = []
    for ctx in _contexts(specs):
        single.append(ctx.run())
        ctx.close()
    ctxs = _contexts(specs)
    res = swig.run_batch(ctxs)
    for r1, r2 in zip(single, res):
        assert _same(r1, r2), (r1, r2)
    for ctx in ctxs:
        ctx.close()


def test_batch_errors():
    ctxs = _contexts(_specs()[:1])
    with pytest.raises(swig.SwigError):
        swig.run_batch([ctxs[0], ctxs[0]])
    ctxs[0].close()
