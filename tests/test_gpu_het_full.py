"""The heterodyned sampler (Sec. 3.4) on the full-size 128 s H1/L1/V1 workload,
through the C-ABI, with every one of the twelve parameters sampled.

The blocks {d_L}, {iota} and {psi} only move the projection factors C_i, so
the sampler evaluates their proposals from the chain's cached per-detector
sums (Z_i / C_i and <h|h>_i / |C_i|^2 of its last full evaluation; the
heterodyned Z_i is linear and <h|h>_i quadratic in C_i).  Here the sky, t_c
and the intrinsic parameters are sampled too, so cached and full evaluations
alternate along every chain.

* Dead and final live points: the logL the sampler reports equals the
  oracle's heterodyned logL of the reported parameters (same fiducial, bins
  and spacing), with the cache and with it switched off.
"""
import numpy as np
import pytest

import parity
import swig_inputs as si
from oracle import events, pp
from oracle import likelihood as L

pytestmark = pytest.mark.gpu

swig = pytest.importorskip("paper_2607_28265_gb300.swig")

NB = 5000
ITERS = 40


# Parity bound: the stated 1e-6 |logL| + 1e-6 (the relative term is ~0.78 here).


@pytest.fixture(scope="module")
def cfg2():
    wl = si.config2()
    ev, th = events.build_event(wl)
    het = L.het_setup(ev, th, NB, spacing="phase")
    return wl, ev, th, het


def _run(wl, ev, th, cache_off, seed=41):
    ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
    ctx.set_sampler(nlive=1000, nrep=100, steps_per_dim=5, seed=seed, likelihood=swig.LIKE_HET, het_bins=NB,
                    het_spacing=0, het_fiducial=th, max_iter=ITERS, cache_off=cache_off)
    r = ctx.run()
    thd, ll, lw = ctx.get_samples()
    ctx.close()
    return r, thd, ll, lw


@pytest.mark.parametrize("cache_off", [0, 1])
def test_full_size_het_dead_points_match_oracle(cfg2, cache_off):
    wl, ev, th, het = cfg2
    assert len(wl.sampled()) == 12
    r, thd, ll, lw = _run(wl, ev, th, cache_off)
    assert r.n_iter >= ITERS and r.n_dead == len(ll)
    # the last 1000 samples are the final live points, all made by chains
    rng = np.random.default_rng(cache_off)
    idx = np.concatenate([rng.choice(len(ll) - 1000, 6, replace=False),
                          len(ll) - 1000 + rng.choice(1000, 10, replace=False)])
    want = np.array([L.het_loglike(ev, het, thd[i]) for i in idx])
    parity.check(f"heterodyned sampler dead points (128 s HLV, cache_off={cache_off})", ll[idx], want, 1e-6, 1e-6)
