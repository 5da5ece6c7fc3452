"""Pins of the oracle's time marginalisation (Sec. 3.1, App. A): t_c summed over
a midpoint grid of time shifts, on the full frequency grid and on the
heterodyned bins.

Each check reaches the oracle from outside: the full-grid overlap as a
function of the shift is a discrete Fourier transform of the per-bin products
(numpy's FFT); the overlap of a noise-free injection peaks at the injected
time; the grid integral of a noise-free injection matches the Laplace form
from the Fisher width of t_c; one node reduces to the plain likelihood; zero
data reduce the marginal to -<h|h>/2; the heterodyned sum tracks the full one;
the grid draw is the inverse CDF on tiny inputs.
"""
import math

import numpy as np
import pytest

import swig_inputs as si
from oracle import events
from oracle import likelihood as L

TC = si.IDX["tc"]


def _params(wl, lo=-0.1, hi=0.1, phase_marg=False):
    params = list(wl.params)
    params[TC] = si.Param(si.PRIOR_UNIFORM, lo, hi, si.MODE_MARG)
    if phase_marg:
        params[si.IDX["phic"]] = si.Param(si.PRIOR_UNIFORM, 0.0, 2 * math.pi, si.MODE_MARG)
    return params


def _event(ev, params, data=None):
    return L.Event(ev.freqs, ev.df, ev.data if data is None else data, ev.psds, ev.detectors, ev.gmst, params)


@pytest.fixture(scope="module")
def cfg1():
    wl = si.config1()
    ev, th = events.build_event(wl)
    ev0, _ = events.build_event(wl, zero_noise=True)
    return wl, ev, ev0, th


def test_full_grid_overlap_is_a_dft(cfg1):
    """Z(t_m) at t_m = m / (N df) equals exp(-2 pi i k_min m / N) FFT(w)[m],
    w_n = 4 df conj(d_n) h_n(t_c = 0) / S_n (numpy's FFT, negative m wrapped)."""
    wl, ev, _, th = cfg1
    evt = _event(ev, _params(wl))
    df = ev.df
    k_min = int(round(ev.freqs[0] / df))
    N = 8192
    th0 = th.copy()
    th0[TC] = 0.0
    h = L.strains(evt, th0)[0]
    w = 4.0 * df * np.conj(ev.data[0]) * h / ev.psds[0]
    F = np.fft.fft(w, N)
    ms = np.array([0, 1, 5, 37, 200, -1, -3, -150])
    t = ms / (N * df)
    z, _ = L.full_time_overlaps(evt, th, t)
    want = np.exp(-2j * math.pi * k_min * (ms % N) / N) * F[ms % N]
    assert np.allclose(z, want, rtol=0, atol=1e-9 * np.max(np.abs(F)))


def test_overlap_peaks_at_the_injected_time(cfg1):
    """A noise-free injection moved to t_c = 12.3 ms (away from zero, so a
    flipped shift sign would peak at -12.3 ms): |Z(t)| peaks there."""
    wl, _, ev0, th = cfg1
    t_inj = 0.0123
    th_inj = th.copy()
    th_inj[TC] = t_inj
    evt = _event(ev0, _params(wl, phase_marg=True))
    evt.data = L.strains(evt, th_inj)
    t = np.concatenate([t_inj + np.linspace(-2e-3, 2e-3, 401), -t_inj + np.linspace(-2e-3, 2e-3, 41)])
    z, _ = L.full_time_overlaps(evt, th, t)
    assert abs(t[np.argmax(np.abs(z))] - t_inj) <= 1e-5


def test_grid_integral_matches_laplace_form(cfg1):
    """Noise-free injection, phi_c marginalised: near its peak logL(t) is
    |Z(t)| - log sqrt(2 pi |Z|) with |Z(t)| ~ W (1 - 2 pi^2 sigma_f^2 dt^2),
    W = <h|h>, sigma_f^2 the variance of f under the weights 4 df |h|^2 / S.
    The grid average over the prior window T is then
    logL(t_inj) + log(sqrt(2 pi) sigma_t / T), sigma_t = 1 / (2 pi sigma_f sqrt(W))."""
    wl, _, ev0, th = cfg1
    params = _params(wl, -0.1, 0.1, phase_marg=True)
    evt = _event(ev0, params)
    h = L.strains(evt, th)[0]
    wgt = 4.0 * ev0.df * np.abs(h) ** 2 / ev0.psds[0]
    W = float(np.sum(wgt))
    f = ev0.freqs
    mean = float(np.sum(wgt * f)) / W
    var = float(np.sum(wgt * f * f)) / W - mean * mean
    sigma_t = 1.0 / (2 * math.pi * math.sqrt(var) * math.sqrt(W))
    assert 2e-5 < sigma_t < 2e-4
    n_nodes = 4000  # 50 us spacing, well inside sigma_t
    got = L.loglike_time_marg_full(evt, th, n_nodes)
    peak = L.loglike(_event(ev0, list(wl.params[:TC]) + [wl.params[TC]] + [params[12]]), th)
    want = peak + math.log(math.sqrt(2 * math.pi) * sigma_t / 0.2)
    assert abs(got - want) < 0.02, (got, want)


def test_one_node_reduces_to_the_plain_likelihood(cfg1):
    wl, ev, _, th = cfg1
    t_mid = 0.0123
    params = _params(wl, t_mid - 1e-3, t_mid + 1e-3)
    plain = list(wl.params)
    th1 = th.copy()
    th1[TC] = t_mid
    got = L.loglike_time_marg_full(_event(ev, params), th, 1)
    want = L.loglike(_event(ev, plain), th1)
    assert abs(got - want) <= 1e-9 * abs(want)
    # heterodyned: a single node at the fiducial's t_c is the heterodyned logL there
    fid = th.copy()
    het = L.het_setup(_event(ev, params), fid, 300, spacing="geometric")
    params_h = _params(wl, fid[TC] - 1e-3, fid[TC] + 1e-3)
    theta = th.copy()
    theta[0] *= 1.0 + 2e-5
    got = L.het_loglike_time_marg(_event(ev, params_h), het, theta, 1)
    theta[TC] = fid[TC]
    want = L.het_loglike(_event(ev, plain), het, theta)
    assert abs(got - want) <= 1e-9 * abs(want)


def test_zero_data_gives_minus_half_hh(cfg1):
    """d = 0: every node has Z = 0, so the grid average is exp(-<h|h>/2)
    exactly and the 1/N_t weights must sum to one."""
    wl, ev, _, th = cfg1
    params = _params(wl, phase_marg=True)
    zero = [np.zeros_like(d) for d in ev.data]
    evz = _event(ev, params, zero)
    hh = L.optimal_snr_sq(evz, th)
    for n in (1, 7, 64):
        assert abs(L.loglike_time_marg_full(evz, th, n) + 0.5 * hh) <= 1e-9 * hh


def test_heterodyned_sum_tracks_the_full_grid(cfg1):
    """Near the fiducial the heterodyned marginal is within ~5e-5 of the
    full-grid one; 5e-4 still fails a flipped A1 term (2e-3 .. 2e-2 here) or
    r0 taken at the left edge instead of the centre (up to 4e-3)."""
    wl, ev, _, th = cfg1
    params = _params(wl, phase_marg=True)
    evt = _event(ev, params)
    het = L.het_setup(evt, th, 450, spacing="geometric")
    rng = np.random.default_rng(5)
    for _ in range(3):
        theta = th.copy()
        theta[0] *= 1.0 + 1e-5 * rng.standard_normal()
        theta[1] = min(1.0, theta[1] * (1.0 + 1e-3 * rng.standard_normal()))
        got = L.het_loglike_time_marg(evt, het, theta, 800)
        want = L.loglike_time_marg_full(evt, theta, 800)
        assert abs(got - want) < 5e-4, (got, want)


def test_draw_time_node_is_the_inverse_cdf():
    w = np.log([1.0, 2.0, 3.0, 4.0])  # cumulative 0.1, 0.3, 0.6, 1.0
    cases = {0.0: 0, 0.05: 0, 0.1: 0, 0.1000001: 1, 0.3: 1, 0.45: 2, 0.6: 2, 0.61: 3, 0.999999: 3}
    for q, j in cases.items():
        assert L.draw_time_node(w, q) == j, q
    # q on a fine uniform grid lands on each node in proportion to its weight
    qs = (np.arange(100000) + 0.5) / 100000
    counts = np.bincount([L.draw_time_node(w, q) for q in qs[::10]], minlength=4)
    assert np.array_equal(counts, [1000, 2000, 3000, 4000])
    # a shift of every log weight changes nothing away from the exact boundaries
    inner = {q: j for q, j in cases.items() if q not in (0.1, 0.3, 0.6)}
    assert all(L.draw_time_node(w + 700.0, q) == j for q, j in inner.items())


def test_time_grid_is_the_midpoint_rule():
    wl = si.config1()
    t = L.time_grid(_params(wl, -0.1, 0.1), 4)
    assert np.allclose(t, [-0.075, -0.025, 0.025, 0.075], atol=1e-15)
    with pytest.raises(ValueError):
        bad = list(wl.params)
        bad[TC] = si.Param(si.PRIOR_SINE, 0.0, 1.0, si.MODE_MARG)
        L.time_grid(bad, 3)


def test_collapsed_edge_sum_equals_the_binned_overlap():
    """The form the device evaluates: with hat weights
    g_ie = [A0_ib/2 - A1_ib/w_b]_(b = e) + [A0_ib/2 + A1_ib/w_b]_(b = e - 1) and
    y_e = sum_i g_ie r_i(e) (ratios at the fiducial's t_c), the overlap at a
    shift dt is sum_e y_e exp(-2 pi i f_e dt); it must equal the per-bin
    heterodyned overlap of the template moved by dt (128 s, H1/L1/V1)."""
    from oracle import physics
    wl = si.config2()
    ev, th = events.build_event(wl)
    params = _params(wl, phase_marg=True)
    evt = _event(ev, params)
    het = L.het_setup(evt, th, 1000)
    theta = th.copy()
    theta[0] *= 1.0 + 3e-6
    theta[si.IDX["ra"]] += 0.01
    nodes = th[TC] + np.array([-2e-3, -1e-4, 0.0, 3e-5, 7e-4])
    z_bins, _ = L.het_time_overlaps(evt, het, theta, nodes)
    w = het.edges[1:] - het.edges[:-1]
    th_ref = theta.copy()
    th_ref[TC] = th[TC]
    th_ref[si.IDX["phic"]] = 0.0
    y = np.zeros(het.edges.size, complex)
    for i, det in enumerate(evt.detectors):
        r = physics.detector_strain(het.edges, th_ref, det, evt.gmst) / het.h0_edges[i]
        g = np.zeros(het.edges.size, complex)
        g[:-1] += 0.5 * het.A0[i] - het.A1[i] / w
        g[1:] += 0.5 * het.A0[i] + het.A1[i] / w
        y += g * r
    z_edges = np.array([np.sum(y * np.exp(-2j * math.pi * het.edges * (t - th[TC]))) for t in nodes])
    assert np.allclose(z_edges, z_bins, rtol=1e-11, atol=1e-9 * np.max(np.abs(z_bins)))
