"""Pins of the oracle likelihood (Eq. 2), phase marginalisation and heterodyning."""
import math

import numpy as np
import pytest
from scipy import integrate

import swig_inputs as si
from oracle import events, physics
from oracle import likelihood as L


@pytest.fixture(scope="module")
def cfg1_zero_noise():
    return events.build_event(si.config1(), zero_noise=True)


@pytest.fixture(scope="module")
def cfg1_noisy():
    return events.build_event(si.config1())


def test_zero_noise_maximum_at_injection(cfg1_zero_noise):
    ev, th = cfg1_zero_noise
    assert L.loglike(ev, th) == pytest.approx(0.0, abs=1e-9)
    rng = np.random.default_rng(3)
    for _ in range(20):
        t2 = th.copy()
        t2[0] *= 1 + rng.normal(0, 1e-4)
        t2[6] *= 1 + rng.normal(0, 0.05)
        t2[11] += rng.normal(0, 1e-3)
        assert L.loglike(ev, t2) < 0.0


def test_inner_product_symmetry_linearity_positivity(cfg1_noisy):
    ev, th = cfg1_noisy
    h = L.strains(ev, th)[0]
    d, s = ev.data[0], ev.psds[0]
    a, b = 0.3 + 0.2j, -1.7
    assert L.inner_product(d, h, s, ev.df) == pytest.approx(L.inner_product(h, d, s, ev.df), rel=1e-13)
    lhs = L.inner_product(d, a * h + b * d, s, ev.df)
    rhs = float(np.real(a * L.complex_overlap(d, h, s, ev.df))) + b * L.inner_product(d, d, s, ev.df)
    assert lhs == pytest.approx(rhs, rel=1e-12)
    assert L.inner_product(h, h, s, ev.df) > 0
    # noise realisation: <n|n> ~ 2 per bin (Re, Im ~ N(0, S/(4 df)))
    n = d - h
    nn = L.inner_product(n, n, s, ev.df) / ev.freqs.size
    assert abs(nn - 2.0) < 5 * 2.0 / math.sqrt(ev.freqs.size)


def test_optimal_snr_against_quadrature(cfg1_noisy):
    """rho^2 = 4 int |h|^2 / S df by adaptive quadrature of the continuous
    integrand vs the oracle's Riemann sum with the Euler-Maclaurin endpoint
    correction df/2 (g(f_lo) + g(f_hi))."""
    ev, th = cfg1_noisy
    det = ev.detectors[0]
    fp, fx = physics.antenna_patterns(det.D, th[9], th[10], th[8], ev.gmst)
    ci = math.cos(th[7])
    q2 = abs(fp * 0.5 * (1 + ci * ci) - 1j * fx * ci) ** 2
    amp2 = physics.amplitude_prefactor(th[0], th[6]) ** 2 * q2
    g = lambda f: 4.0 * amp2 * f ** (-7.0 / 3.0) / si.design_psd(np.array([f]))[0]
    lo, hi = ev.freqs[0], ev.freqs[-1]
    val, err = integrate.quad(g, lo, hi, limit=400, epsrel=1e-12)
    riemann = L.optimal_snr_sq(ev, th)
    corrected = riemann - 0.5 * ev.df * (g(lo) + g(hi))
    assert corrected == pytest.approx(val, rel=1e-5)


def test_phase_marginalisation_matches_brute_force_grid():
    wl = si.config1()
    wl.params[si.IDX["phic"]] = si.Param(si.PRIOR_UNIFORM, 0.0, 2 * math.pi, mode=si.MODE_MARG)
    ev, th = events.build_event(wl)
    for dt in (0.0, 2e-4, -1e-3):
        t2 = th.copy(); t2[11] += dt
        assert L.loglike(ev, t2) == pytest.approx(L.loglike_phase_grid(ev, t2, 4096), abs=1e-8)


def test_heterodyne_exact_at_fiducial_and_converges(cfg1_noisy):
    ev, th = cfg1_noisy
    full = L.loglike(ev, th)
    errs = []
    for nb in (150, 300, 600):
        het = L.het_setup(ev, th, nb)
        assert L.het_loglike(ev, het, th) == pytest.approx(full, rel=1e-12, abs=1e-9)
        t2 = th.copy(); t2[0] *= 1 + 2e-4; t2[11] += 3e-4
        errs.append(abs(L.het_loglike(ev, het, t2) - L.loglike(ev, t2)))
    # linear-in-bin ratio: error falls roughly like (bin width)^2
    assert errs[1] < errs[0] and errs[2] < errs[1]
    assert errs[2] < 0.05


def test_het_phase_edges_cover_grid(cfg1_noisy):
    ev, _ = cfg1_noisy
    edges, idx = L.phase_bound_edges(ev.freqs, 300)
    assert edges[0] == ev.freqs[0] and edges[-1] == ev.freqs[-1]
    assert np.all(np.diff(idx) > 0)
    # equal increments of the phase-bound function, before snapping to the grid
    assert 250 <= edges.size - 1 <= 300


def test_heterodyne_is_second_order_for_an_amplitude_varying_template(cfg1_noisy, monkeypatch):
    """Summary-data signs (A1, B1) against the exact inner products.

    Every template of this model has |h / h0| constant in f, and then
    Re(r0 r1*) = (|r_hi|^2 - |r_lo|^2) / (2 w) = 0 in every bin, so B1 never
    contributes.  To fix its sign the template here is the fiducial times a
    real amplitude ramp a(f) = 1 + eps (f - f_ref) / f_ref, which is linear in
    f, so r is exactly linear in each bin.  Then, from the definitions:
    * Z = sum_b (A0 r0 + A1 r1) equals the full-grid 4 df sum d* h / S to
      rounding (Z is linear in r);
    * <h|h>_het = sum_b (B0 |r0|^2 + 2 B1 Re(r0 r1*)) misses only
      sum_b |r1|^2 sum_(f in b) |h0|^2 w (f - f_c)^2 >= 0, which is second order
      in eps: the error is negative and quadruples when eps doubles.  A B1 of
      the wrong sign leaves a first-order error (the ratio would be ~2)."""
    ev, th = cfg1_noisy
    het = L.het_setup(ev, th, 300, spacing="phase")
    f_ref = 100.0
    base = physics.detector_strain
    errs = []
    for eps in (0.01, 0.02):
        def ramp(f, theta, det, gmst, eps=eps):
            return base(f, theta, det, gmst) * (1.0 + eps * (np.asarray(f) - f_ref) / f_ref)

        monkeypatch.setattr(physics, "detector_strain", ramp)
        z_het, hh_het = L.het_overlap(ev, het, th)
        h = L.strains(ev, np.asarray(th))
        monkeypatch.setattr(physics, "detector_strain", base)
        z_ex = sum(L.complex_overlap(d, hi, s, ev.df) for d, hi, s in zip(ev.data, h, ev.psds))
        hh_ex = sum(L.inner_product(hi, hi, s, ev.df) for hi, s in zip(h, ev.psds))
        assert abs(z_het - z_ex) <= 1e-10 * abs(z_ex)
        errs.append(hh_het - hh_ex)
    assert errs[0] < 0.0 and errs[1] < 0.0
    assert errs[1] / errs[0] == pytest.approx(4.0, rel=0.02)
    assert abs(errs[1]) < 1e-4 * hh_ex
