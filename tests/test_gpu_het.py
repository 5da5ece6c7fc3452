"""Heterodyned likelihood (Sec. 3.4) on the GPU against the oracle's het_loglike.

The library forms the bin edges, the fiducial waveform and the summary data
itself; the oracle forms its own (FP64, numpy).  Both must give the same
heterodyned logL for the same fiducial, bin count and spacing.  The device
contraction is FP32 per bin: its rounding error is bounded by a few ulps of
the sum of the absolute per-bin terms, which here never exceeds ~2x the
matched-filter SNR^2 plus <h|h> (the constant -<d|d>/2 is FP64 on both sides).
The checks use the stated parity bound 1e-6 |logL| + 1e-6: with -<d|d>/2 in
logL the relative term dominates (~4e-3 on the 4 s grid, where the largest
measured error is 1.7e-3).
"""
import numpy as np
import pytest

import parity
import swig_inputs as si
from oracle import events
from oracle import likelihood as L

pytestmark = pytest.mark.gpu

swig = pytest.importorskip("paper_2607_28265_gb300.swig")


def _tol(want):
    # the heterodyne against the full grid at the injection (an approximation
    # error, not a parity bound)
    return 1e-6 * np.abs(want) + 2e-4


def _ctx(wl, ev, params=None):
    ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
    if params is not None:
        ctx.set_prior(params)
    return ctx


def _thetas(wl, ev, th_inj, n, seed, spread):
    """Prior draws and points near the injection (spread in unit-cube units)."""
    rng = np.random.default_rng(seed)
    sampled = wl.sampled()
    from oracle import physics
    u_prior = rng.random((n, len(sampled)))
    far = physics.prior_transform(u_prior, wl.params)
    # near: small perturbations of the injection, mapped back through the prior
    lo = np.array([wl.params[s].lo for s in sampled])
    hi = np.array([wl.params[s].hi for s in sampled])
    near = np.repeat(th_inj[None, :], n, axis=0)
    for j, s in enumerate(sampled):
        p = wl.params[s]
        if p.kind == si.PRIOR_UNIFORM:
            near[:, s] = np.clip(th_inj[s] + spread * (hi[j] - lo[j]) * rng.standard_normal(n), lo[j], hi[j])
    return np.concatenate([far, near])


@pytest.fixture(scope="module")
def cfg1():
    wl = si.config1()
    ev, th = events.build_event(wl)
    return wl, ev, th


@pytest.mark.parametrize("n_bins", [300, 450, 600])
def test_het_matches_oracle_cfg1(cfg1, n_bins):
    wl, ev, th = cfg1
    het = L.het_setup(ev, th, n_bins)
    ctx = _ctx(wl, ev)
    ctx.set_sampler(nlive=100, nrep=10, likelihood=swig.LIKE_HET, het_bins=n_bins, het_fiducial=th)
    thetas = _thetas(wl, ev, th, 40, n_bins, 0.002)
    got = ctx.loglike_batch(thetas)
    want = np.array([L.het_loglike(ev, het, t) for t in thetas])
    parity.check(f"heterodyned batch (4 s H1, {n_bins} bins)", got, want, 1e-6, 1e-6)
    # at the fiducial itself the heterodyned logL is the full logL up to the
    # FP32 contraction (r = 1 exactly in every bin)
    full = L.loglike(ev, th)
    assert abs(ctx.loglike_batch(th[None, :])[0] - full) <= _tol(full)
    ctx.close()


def test_het_geometric_spacing_and_fiducial_offset(cfg1):
    """Geometric edges and a fiducial away from the injection."""
    wl, ev, th = cfg1
    fid = th.copy()
    fid[si.IDX["mc"]] += 1e-4
    fid[si.IDX["tc"]] += 2e-4
    het = L.het_setup(ev, fid, 400, spacing="geometric")
    ctx = _ctx(wl, ev)
    ctx.set_sampler(nlive=100, nrep=10, likelihood=swig.LIKE_HET, het_bins=400, het_spacing=1, het_fiducial=fid)
    thetas = _thetas(wl, ev, th, 30, 99, 0.003)
    got = ctx.loglike_batch(thetas)
    want = np.array([L.het_loglike(ev, het, t) for t in thetas])
    parity.check("heterodyned batch (4 s H1, geometric, offset fiducial)", got, want, 1e-6, 1e-6)
    ctx.close()


def test_het_full_size_three_detectors():
    """128 s H1/L1/V1 grid (259,585 bins per detector), phase marginalised,
    1000 bins, fiducial at the injection."""
    wl = si.config2()
    ev, th = events.build_event(wl)
    het = L.het_setup(ev, th, 1000)
    ctx = _ctx(wl, ev)
    ctx.set_sampler(nlive=1000, nrep=100, likelihood=swig.LIKE_HET, het_bins=1000, het_fiducial=th)
    thetas = _thetas(wl, ev, th, 24, 5, 0.0005)
    got = ctx.loglike_batch(thetas)
    want = np.array([L.het_loglike(ev, het, t) for t in thetas])
    parity.check("heterodyned batch (128 s HLV, 5000 bins)", got, want, 1e-6, 1e-6)
    # switching back to the full likelihood re-prepares the context
    ctx.set_sampler(nlive=1000, nrep=100, likelihood=swig.LIKE_FULL)
    full = ctx.loglike_batch(thetas[-4:])
    want_full = np.array([L.loglike(ev, t) for t in thetas[-4:]])
    parity.check("full-grid batch beside the heterodyned one (128 s HLV)", full, want_full, 1e-6, 1e-6)
    ctx.close()


def test_het_invalid_and_errors(cfg1):
    wl, ev, th = cfg1
    ctx = _ctx(wl, ev)
    with pytest.raises(swig.SwigError):
        ctx.set_sampler(nlive=100, nrep=10, likelihood=swig.LIKE_HET, het_bins=1, het_fiducial=th)
    with pytest.raises(swig.SwigError):
        ctx.set_sampler(nlive=100, nrep=10, likelihood=swig.LIKE_HET, het_bins=100, het_spacing=2, het_fiducial=th)
    bad = th.copy()
    bad[si.IDX["q"]] = 2.0
    ctx.set_sampler(nlive=100, nrep=10, likelihood=swig.LIKE_HET, het_bins=100, het_fiducial=bad)
    with pytest.raises(swig.SwigError) as e:
        ctx.loglike_batch(th[None, :])
    assert e.value.code == swig.SWIG_E_ARG
    ctx.set_sampler(nlive=100, nrep=10, likelihood=swig.LIKE_HET, het_bins=100, het_fiducial=th)
    t = np.repeat(th[None, :], 3, axis=0)
    t[1, si.IDX["q"]] = 1.5  # outside q <= 1: -inf like the full likelihood
    got = ctx.loglike_batch(t)
    assert np.isfinite(got[0]) and got[1] == -np.inf and got[0] == got[2]
    ctx.close()
