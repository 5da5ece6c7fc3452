"""The sampler with the learned slice proposal on the 4 s single-detector
workload, through the C-ABI: dead points against the oracle likelihood,
determinism, and evidence/posterior against the same references as plain
SwiG (plain SwiG is the reference for correctness)."""
import math
import os

import numpy as np
import pytest

import parity
import swig_inputs as si
from oracle import events, pp
from oracle import likelihood as L

pytestmark = pytest.mark.gpu

swig = pytest.importorskip("paper_2607_28265_gb300.swig")

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def cfg1():
    wl = si.config1()
    ev, th = events.build_event(wl)
    return wl, ev, th


def _run(wl, ev, nlive, nrep, seed, proposal, **kw):
    ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
    ctx.set_sampler(nlive=nlive, nrep=nrep, steps_per_dim=5, seed=seed, precision=swig.PREC_MIXED,
                    proposal=proposal, **kw)
    r = ctx.run()
    thd, ll, lw = ctx.get_samples()
    return ctx, r, thd, ll, lw


def test_learned_dead_points_match_oracle_and_are_deterministic(cfg1):
    wl, ev, th = cfg1
    ctx, r, thd, ll, lw = _run(wl, ev, 200, 20, 11, swig.PROPOSAL_LEARNED)
    prof = ctx.profile()
    assert prof["learn_rounds"] >= 2 and prof["learn_ms"] > 0
    assert r.status == 0 and np.isfinite(r.logz)
    m = lw.max()
    assert abs(m + math.log(np.sum(np.exp(lw - m))) - r.logz) < 1e-9
    idx = np.linspace(0, len(ll) - 1, 16).astype(int)
    want = np.array([L.loglike(ev, thd[i]) for i in idx])
    parity.check("learned-proposal sampler dead points (4 s H1)", ll[idx], want, 1e-6, 1e-6)
    r2 = ctx.run()
    thd2, ll2, _ = ctx.get_samples()
    assert r2.logz == r.logz and np.array_equal(ll, ll2) and np.array_equal(thd, thd2)
    ctx.close()


def test_learned_posterior_and_evidence(cfg1):
    isf = os.path.join(HERE, "golden", "cfg1_is_evidence.txt")
    logz_true = float(open(isf).readlines()[-1].split()[0])
    post = os.path.join(HERE, "golden", "cfg1_is_posterior.csv")
    ref_logz = float(open(post).readlines()[1].split("logz=")[1].split()[0])
    ref = np.loadtxt(post, delimiter=",", comments="#", skiprows=3)
    wl, ev, th = cfg1
    zs = []
    for seed in (5, 6, 7, 8):
        ctx, r, thd, ll, lw = _run(wl, ev, 400, 40, seed, swig.PROPOSAL_LEARNED)
        zs.append(r.logz)
        if seed == 5:
            for j, slot in enumerate(wl.sampled()):
                d, p = pp.weighted_ks_2samp(thd[:, slot], np.exp(lw - r.logz), ref[:, j],
                                            np.exp(ref[:, -1] - ref_logz))
                assert p > 1e-3, (si.PARAM_NAMES[slot], d, p)
        ctx.close()
    assert abs(np.mean(zs) - logz_true) < 2.0, (zs, logz_true)
