"""Pins of the oracle's distance marginalisation (Sec. 3.1) against special
cases, brute-force quadrature and the plain likelihood."""
import math

import numpy as np
import pytest

import swig_inputs as si
from oracle import events, physics
from oracle import likelihood as L

P2 = si.Param(si.PRIOR_POWER2, 30.0, 150.0, si.MODE_MARG)
PU = si.Param(si.PRIOR_UNIFORM, 20.0, 200.0, si.MODE_MARG)


def test_no_signal_gives_data_term():
    for p in (P2, PU):
        for pm in (False, True):
            assert L.log_distance_integral(0.0j, 0.0, 1234.5, p, pm) == pytest.approx(-617.25, abs=1e-10)


def test_point_prior_reduces_to_plain_likelihood():
    z1, h1 = 4.0e4 + 1.0e4j, 1.7e7
    d = 80.0
    p = si.Param(si.PRIOR_UNIFORM, d, d * (1 + 1e-11), si.MODE_MARG)  # logL changes by ~2e-8 across it
    for pm in (False, True):
        want = float(L.loglike_at_distance(z1, h1, 10.0, d, pm))
        assert L.log_distance_integral(z1, h1, 10.0, p, pm) == pytest.approx(want, abs=1e-6)


@pytest.mark.parametrize("p", [P2, PU])
def test_against_brute_force_riemann_sum(p):
    """Midpoint sum with 4e6 cells (error ~ h^2 f'' / 24, far below 1e-8)."""
    z1, h1, dd = 6.0e4 - 2.0e4j, 4.0e7, 50.0
    n = 4_000_000
    h = (p.hi - p.lo) / n
    d = p.lo + h * (np.arange(n) + 0.5)
    for pm in (False, True):
        lg = L.loglike_at_distance(z1, h1, dd, d, pm) + np.log(L.distance_prior_pdf(d, p))
        m = lg.max()
        brute = m + math.log(np.sum(np.exp(lg - m)) * h)
        assert L.log_distance_integral(z1, h1, dd, p, pm) == pytest.approx(brute, abs=1e-8)


def test_phase_and_distance_against_nested_grid():
    """Both marginals by brute force: uniform phase grid (exact for the
    trigonometric integrand to rounding) inside a fine distance grid."""
    z1, h1, dd = 3.0e4 + 2.5e4j, 3.0e7, 5.0
    p = PU
    nd, nphi = 200_000, 512
    h = (p.hi - p.lo) / nd
    d = p.lo + h * (np.arange(nd) + 0.5)
    phis = 2 * math.pi * np.arange(nphi) / nphi
    acc = np.zeros(nd)
    # logL(d, phi) = Re(z1 e^{i phi}) / d - h1 / (2 d^2) - dd / 2
    base = -0.5 * h1 / d ** 2 - 0.5 * dd
    lmax = np.abs(z1) / d + base
    for ph in phis:
        acc += np.exp(np.real(z1 * np.exp(1j * ph)) / d + base - lmax)
    lg = lmax + np.log(acc / nphi) + np.log(L.distance_prior_pdf(d, p))
    m = lg.max()
    brute = m + math.log(np.sum(np.exp(lg - m)) * h)
    assert L.log_distance_integral(z1, h1, dd, p, True) == pytest.approx(brute, abs=1e-6)


def test_amplitude_law_matches_full_likelihood():
    """logL(theta with d_L = d) from the waveform itself equals the 1/d
    scaling of the 1 Mpc overlaps used by the marginal."""
    wl = si.config1()
    ev, th = events.build_event(wl)
    t1 = th.copy()
    t1[si.IDX["dl"]] = 1.0
    z1, h1, dd = L.overlaps_at(ev, t1)
    for d in (25.0, 80.0, 190.0):
        t = th.copy()
        t[si.IDX["dl"]] = d
        want = L.loglike(ev, t)
        got = float(L.loglike_at_distance(z1, h1, dd, d, False))
        assert got == pytest.approx(want, rel=1e-12, abs=1e-9)


def test_quantiles_without_signal_are_prior_quantiles():
    for p in (P2, PU):
        for u in (0.05, 0.5, 0.93):
            want = float(physics.prior_transform_1d(u, p.kind, p.lo, p.hi))
            assert L.distance_quantile(0.0j, 0.0, 0.0, p, False, u) == pytest.approx(want, abs=1e-8)


def test_event_dispatch_and_dead_point_draw():
    """An event whose d_L slot is marginalised routes loglike() to the
    marginal; a drawn distance lies inside the prior and near the peak."""
    wl = si.config1()
    ev, th = events.build_event(wl)
    params = list(ev.params)
    params[si.IDX["dl"]] = si.Param(si.PRIOR_UNIFORM, 20.0, 200.0, si.MODE_MARG)
    evm = L.Event(ev.freqs, ev.df, ev.data, ev.psds, ev.detectors, ev.gmst, params)
    v = L.loglike(evm, th)
    t1 = th.copy()
    t1[si.IDX["dl"]] = 1.0
    z1, h1, dd = L.overlaps_at(evm, t1)
    assert v == pytest.approx(L.log_distance_integral(z1, h1, dd, params[si.IDX["dl"]], False), abs=1e-12)
    d50 = L.draw_distance(evm, th, 0.5)
    assert 20.0 < d50 < 200.0 and abs(d50 - th[si.IDX["dl"]]) < 30.0
