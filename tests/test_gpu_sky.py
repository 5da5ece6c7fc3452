"""Detector-frame sky parameterisation on the GPU: the prior transform
against the oracle's, and the sampler on a two-detector 4 s workload with the
sky free, whose evidence must equal that of the equatorial parameterisation
(same isotropic prior; compared as two samples of runs) and whose dead points
match the oracle likelihood."""
import math

import numpy as np
import pytest

import parity
import swig_inputs as si
from oracle import events, physics
from oracle import likelihood as L

pytestmark = pytest.mark.gpu

swig = pytest.importorskip("paper_2607_28265_gb300.swig")


def _workload(frame):
    wl = si.config1()
    wl.detectors = ("H1", "L1")
    wl.params[si.IDX["ra"]] = (si.Param(si.PRIOR_UNIFORM, 0.0, 2 * math.pi, block=3) if frame else
                               si.Param(si.PRIOR_UNIFORM, 0.0, 2 * math.pi, block=3))
    wl.params[si.IDX["dec"]] = (si.Param(si.PRIOR_SINE, 0.0, math.pi, block=3) if frame else
                                si.Param(si.PRIOR_COSINE, -math.pi / 2, math.pi / 2, block=3))
    return wl


def test_prior_transform_matches_oracle():
    wl = _workload(True)
    ev, th = events.build_event(wl)
    ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
    ctx.set_sky_frame(0, 1)
    u = np.random.default_rng(3).random((64, len(wl.sampled())))
    got = ctx.prior_transform(u)
    va, _, _ = si.site_vectors("H1")
    vb, _, _ = si.site_vectors("L1")
    want = physics.prior_transform(u, wl.params, sky=(physics.detector_frame(va, vb), ev.gmst))
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
    # a prior that does not fit the frame is refused when used
    bad = list(wl.params)
    bad[si.IDX["dec"]] = si.Param(si.PRIOR_COSINE, -math.pi / 2, math.pi / 2, block=3)
    ctx.set_prior(bad)
    with pytest.raises(swig.SwigError):
        ctx.prior_transform(u)
    ctx.close()


def test_sampler_evidence_matches_equatorial():
    zs = {}
    for frame in (True, False):
        wl = _workload(frame)
        ev, th = events.build_event(_workload(False))  # same data for both
        runs = []
        for seed in (51, 52, 53, 54, 55, 56):
            ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
            if frame:
                ctx.set_sky_frame(0, 1)
            ctx.set_sampler(nlive=400, nrep=40, steps_per_dim=5, seed=seed, precision=swig.PREC_MIXED)
            r = ctx.run()
            thd, ll, lw = ctx.get_samples()
            runs.append(r.logz)
            if seed == 51:
                idx = np.linspace(0, len(ll) - 1, 8).astype(int)
                want = np.array([L.loglike(ev, thd[i]) for i in idx])
                parity.check("detector-frame sky sampler dead points", ll[idx], want, 1e-6, 1e-6)
                assert np.all((thd[:, si.IDX["dec"]] >= -math.pi / 2) & (thd[:, si.IDX["dec"]] <= math.pi / 2))
            ctx.close()
        zs[frame] = runs
    # single runs scatter by ~1-2 nats here (the sky ring of two detectors mixes
    # slowly), so the means are compared at three combined standard errors
    a, b = np.array(zs[True]), np.array(zs[False])
    se = math.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
    assert abs(a.mean() - b.mean()) < 3.0 * se + 0.3, zs
