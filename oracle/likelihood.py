"""Matched-filter log-likelihood in FP64 (Sec. 3.1, Eq. 2), its phase-,
distance- and time-marginalised forms (Sec. 3.1, App. A) and its heterodyned
approximation (Sec. 3.4).

Event layout: an ``Event`` holds the frequency grid, per-detector data d_i(f),
PSDs S_i(f), detector geometry, GMST and the prior description.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import i0e

from scipy import integrate

from swig_inputs import IDX, MODE_MARG, MODE_SAMPLE, PRIOR_POWER2, PRIOR_UNIFORM
from . import physics


@dataclass
class Event:
    freqs: np.ndarray
    df: float
    data: list          # complex arrays, one per detector
    psds: list          # real arrays, one per detector
    detectors: list     # physics.Detector
    gmst: float
    params: list        # swig_inputs.Param, 13 slots

    @property
    def phase_marginalised(self) -> bool:
        return self.params[IDX["phic"]].mode == MODE_MARG

    @property
    def distance_marginalised(self) -> bool:
        return self.params[IDX["dl"]].mode == MODE_MARG


def inner_product(a, b, psd, df):
    """<a|b> = 4 Re int a* b / S df, as the Riemann sum over the grid (Sec. 3.1)."""
    return 4.0 * df * float(np.real(np.sum(np.conj(a) * b / psd)))


def complex_overlap(a, b, psd, df):
    """4 df sum a* b / S without taking the real part."""
    return 4.0 * df * complex(np.sum(np.conj(a) * b / psd))


def strains(ev: Event, theta):
    return [physics.detector_strain(ev.freqs, theta, det, ev.gmst) for det in ev.detectors]


def loglike(ev: Event, theta):
    """Eq. 2: logL = -1/2 sum_i <d_i - h_i | d_i - h_i>_i.

    With phi_c marginalised (Sec. 3.1) over U[0, 2 pi):
        logL = log I0(|Z|) - 1/2 sum_i <h_i|h_i> - 1/2 sum_i <d_i|d_i>,
        Z = sum_i 4 df sum_f d_i* h_i / S_i evaluated at phi_c = 0,
    because the template depends on phi_c only through exp(i phi_c).  The
    normalisation -1/2 sum log(2 pi S) is a constant and is omitted.
    """
    theta = np.asarray(theta, dtype=np.float64)
    if ev.distance_marginalised:
        return loglike_distance_marg(ev, theta)
    if ev.phase_marginalised:
        th = theta.copy()
        th[IDX["phic"]] = 0.0
        hs = strains(ev, th)
        z = sum(complex_overlap(d, h, s, ev.df) for d, h, s in zip(ev.data, hs, ev.psds))
        hh = sum(inner_product(h, h, s, ev.df) for h, s in zip(hs, ev.psds))
        dd = sum(inner_product(d, d, s, ev.df) for d, s in zip(ev.data, ev.psds))
        x = abs(z)
        return x + math.log(i0e(x)) - 0.5 * hh - 0.5 * dd
    hs = strains(ev, theta)
    return -0.5 * sum(inner_product(d - h, d - h, s, ev.df) for d, h, s in zip(ev.data, hs, ev.psds))


def loglike_phase_grid(ev: Event, theta, n_phase=4096):
    """Brute-force phase marginal: log mean_j exp(logL(phi_j)) on a uniform grid.

    Used to pin the closed-form log I0 expression (Sec. 3.1 says the phase may
    equally be marginalised by summation over a dense grid).
    """
    theta = np.asarray(theta, dtype=np.float64).copy()
    theta[IDX["phic"]] = 0.0
    hs = strains(ev, theta)
    dd = sum(inner_product(d, d, s, ev.df) for d, s in zip(ev.data, ev.psds))
    phis = 2.0 * math.pi * np.arange(n_phase) / n_phase
    vals = []
    for phi in phis:
        # exp(-i Psi) with Psi containing -phi_c: template scales by exp(i phi).
        vals.append(-0.5 * sum(inner_product(d - h * np.exp(1j * phi), d - h * np.exp(1j * phi), s, ev.df)
                               for d, h, s in zip(ev.data, hs, ev.psds)))
    vals = np.array(vals)
    m = vals.max()
    return m + math.log(np.mean(np.exp(vals - m)))


# --------------------------------------------------------------------------
# Distance marginalisation (Sec. 3.1; the paper's default injection setting)
# --------------------------------------------------------------------------
def distance_prior_pdf(d, p):
    """Normalised density of the d_L prior family on [lo, hi]."""
    d = np.asarray(d, dtype=np.float64)
    inside = (d >= p.lo) & (d <= p.hi)
    if p.kind == PRIOR_POWER2:
        val = 3.0 * d * d / (p.hi ** 3 - p.lo ** 3)
    elif p.kind == PRIOR_UNIFORM:
        val = np.full_like(d, 1.0 / (p.hi - p.lo))
    else:
        raise ValueError("distance prior must be uniform or power-law 2")
    return np.where(inside, val, 0.0)


def overlaps_at(ev: Event, theta):
    """(Z, H, DD) of template theta: Z = sum_i 4 df sum d_i* h_i / S_i (at
    phi_c = 0 when it is marginalised), H = sum_i <h_i|h_i>, DD = sum_i <d_i|d_i>."""
    th = np.asarray(theta, dtype=np.float64).copy()
    if ev.phase_marginalised:
        th[IDX["phic"]] = 0.0
    hs = strains(ev, th)
    z = sum(complex_overlap(d, h, s, ev.df) for d, h, s in zip(ev.data, hs, ev.psds))
    hh = sum(inner_product(h, h, s, ev.df) for h, s in zip(hs, ev.psds))
    dd = sum(inner_product(d, d, s, ev.df) for d, s in zip(ev.data, ev.psds))
    return z, hh, dd


def loglike_at_distance(z1, h1, dd, d, phase_marg):
    """logL at distance d from the overlaps z1, h1 of the same template at
    d_L = 1 Mpc: the amplitude scales as 1/d_L, so Z(d) = z1 / d and
    <h|h>(d) = h1 / d^2 (Eq. 2 expanded; log I0 form with phi_c marginalised)."""
    d = np.asarray(d, dtype=np.float64)
    if phase_marg:
        x = np.abs(z1) / d
        core = x + np.log(i0e(x))
    else:
        core = np.real(z1) / d
    return core - 0.5 * h1 / (d * d) - 0.5 * dd


def log_distance_integral(z1, h1, dd, p, phase_marg):
    """log int pi(d) L(d) dd over the prior [lo, hi] of slot p, by adaptive
    quadrature around the integrand's peak (located on a dense grid)."""
    grid = np.linspace(p.lo, p.hi, 20001)
    lg = loglike_at_distance(z1, h1, dd, grid, phase_marg) + np.log(distance_prior_pdf(grid, p))
    m = float(np.max(lg))
    d_peak = float(grid[int(np.argmax(lg))])

    def f(d):
        return float(distance_prior_pdf(d, p) * np.exp(loglike_at_distance(z1, h1, dd, d, phase_marg) - m))

    val, _ = integrate.quad(f, p.lo, p.hi, points=[d_peak], limit=500, epsabs=0.0, epsrel=1e-12)
    return m + math.log(val)


def loglike_distance_marg(ev: Event, theta):
    """log of int pi(d_L) L(theta, d_L) d d_L over the d_L prior: the
    likelihood marginalised over distance (the definition, written out)."""
    th = np.asarray(theta, dtype=np.float64).copy()
    th[IDX["dl"]] = 1.0
    z1, h1, dd = overlaps_at(ev, th)
    return log_distance_integral(z1, h1, dd, ev.params[IDX["dl"]], ev.phase_marginalised)


def distance_cdf(z1, h1, dd, p, phase_marg, d):
    """P(d_L <= d | theta, data) under the prior p (the conditional the
    post-hoc reconstruction draws from)."""
    lz = log_distance_integral(z1, h1, dd, p, phase_marg)

    def f(x):
        return float(distance_prior_pdf(x, p) * np.exp(loglike_at_distance(z1, h1, dd, x, phase_marg) - lz))

    if d <= p.lo:
        return 0.0
    val, _ = integrate.quad(f, p.lo, min(d, p.hi), limit=500, epsabs=1e-14, epsrel=1e-12)
    return min(1.0, val)


def distance_quantile(z1, h1, dd, p, phase_marg, u):
    """The u-quantile of p(d_L | theta, data) (root of the conditional CDF)."""
    from scipy.optimize import brentq
    return brentq(lambda d: distance_cdf(z1, h1, dd, p, phase_marg, d) - u, p.lo, p.hi, xtol=1e-10, rtol=1e-12)


def draw_distance(ev: Event, theta, u):
    """Post-hoc d_L of a sample: the u-quantile of p(d_L | theta, data)."""
    th = np.asarray(theta, dtype=np.float64).copy()
    th[IDX["dl"]] = 1.0
    z1, h1, dd = overlaps_at(ev, th)
    return distance_quantile(z1, h1, dd, ev.params[IDX["dl"]], ev.phase_marginalised, u)


def optimal_snr_sq(ev: Event, theta):
    return sum(inner_product(h, h, s, ev.df) for h, s in zip(strains(ev, theta), ev.psds))


def loglike_u(ev: Event, u_sampled):
    """logL at unit-cube coordinates of the sampled parameters (-inf outside)."""
    u = np.asarray(u_sampled, dtype=np.float64)
    if np.any(u < 0.0) or np.any(u > 1.0):
        return -np.inf
    theta = physics.prior_transform(u, ev.params)[0]
    return loglike(ev, theta)


# --------------------------------------------------------------------------
# Heterodyned (relative-binning) likelihood, Sec. 3.4
# --------------------------------------------------------------------------
@dataclass
class Het:
    edges: np.ndarray        # N_b + 1 bin-edge frequencies
    centers: np.ndarray      # N_b bin centres
    A0: list                 # per detector, complex (N_b,)
    A1: list
    B0: list                 # per detector, real (N_b,)
    B1: list
    h0_edges: list           # fiducial strain at the edges, per detector
    theta_fid: np.ndarray


def phase_bound_edges(freqs, n_bins, f_lo=None, f_hi=None):
    """Edges of equal maximum phase change (Zackay, Dai & Venumadhav 2018).

    The maximum dephasing between templates grows like
    g(f) = sum_gamma sign(gamma) (f / f*_gamma)^gamma over the PN power laws
    gamma in {-5/3, -2/3, 1, 5/3, 7/3}, f* = f_lo for negative powers and f_hi
    for positive ones.  Edges split g into n_bins equal increments and are
    snapped to grid frequencies, so every grid bin falls in exactly one bin.
    The exponent set is the construction's heuristic: the pins check the edge
    structure and the heterodyne's accuracy, not the set itself (parity
    unpinned for the exact edge positions; any set gives a valid heterodyne).
    """
    f_lo = freqs[0] if f_lo is None else f_lo
    f_hi = freqs[-1] if f_hi is None else f_hi
    gammas = (-5.0 / 3.0, -2.0 / 3.0, 1.0, 5.0 / 3.0, 7.0 / 3.0)

    def g(f):
        out = np.zeros_like(f)
        for gm in gammas:
            fs = f_lo if gm < 0 else f_hi
            out += np.sign(gm) * (f / fs) ** gm
        return out

    gf = g(freqs)
    targets = np.linspace(gf[0], gf[-1], n_bins + 1)
    idx = np.searchsorted(gf, targets, side="left")
    idx[0], idx[-1] = 0, freqs.size - 1
    idx = np.unique(idx)
    return freqs[idx], idx


def geometric_edges(freqs, n_bins):
    """Optional geometric spacing of edges, snapped to grid frequencies."""
    targets = np.geomspace(freqs[0], freqs[-1], n_bins + 1)
    idx = np.unique(np.clip(np.searchsorted(freqs, targets), 0, freqs.size - 1))
    idx[0], idx[-1] = 0, freqs.size - 1
    return freqs[np.unique(idx)], np.unique(idx)


def het_setup(ev: Event, theta_fid, n_bins, spacing="phase"):
    """Summary data per detector and bin (Sec. 3.4), in FP64.

    Bin b holds the grid bins with edges[b] <= f < edges[b+1] (the last bin also
    holds f = edges[-1]).  With centre f_c = (edges[b] + edges[b+1]) / 2:
        A0 = 4 df sum d* h0 / S,   A1 = 4 df sum d* h0 / S (f - f_c)
        B0 = 4 df sum |h0|^2 / S,  B1 = 4 df sum |h0|^2 / S (f - f_c)
    """
    theta_fid = np.asarray(theta_fid, dtype=np.float64).copy()
    if ev.phase_marginalised:
        theta_fid[IDX["phic"]] = 0.0
    if spacing == "phase":
        edges, idx = phase_bound_edges(ev.freqs, n_bins)
    else:
        edges, idx = geometric_edges(ev.freqs, n_bins)
    nb = edges.size - 1
    # bin index of each grid frequency
    which = np.searchsorted(idx, np.arange(ev.freqs.size), side="right") - 1
    which[-1] = nb - 1
    centers = 0.5 * (edges[:-1] + edges[1:])
    h0s = strains(ev, theta_fid)
    A0, A1, B0, B1, h0e = [], [], [], [], []
    for d, h0, s, det in zip(ev.data, h0s, ev.psds, ev.detectors):
        w = 4.0 * ev.df / s
        dh = np.conj(d) * h0 * w
        hh = np.abs(h0) ** 2 * w
        off = ev.freqs - centers[which]
        A0.append(np.bincount(which, weights=dh.real, minlength=nb) + 1j * np.bincount(which, weights=dh.imag, minlength=nb))
        A1.append(np.bincount(which, weights=(dh * off).real, minlength=nb) + 1j * np.bincount(which, weights=(dh * off).imag, minlength=nb))
        B0.append(np.bincount(which, weights=hh, minlength=nb))
        B1.append(np.bincount(which, weights=hh * off, minlength=nb))
        h0e.append(physics.detector_strain(edges, theta_fid, det, ev.gmst))
    return Het(edges, centers, A0, A1, B0, B1, h0e, theta_fid)


def het_overlap(ev: Event, het: Het, theta):
    """Heterodyned complex overlap Z = sum_i sum_b (A0 r0 + A1 r1) and <h|h>.

    r = h/h0 at the edges, taken linear in each bin: r0 the mean of the two
    edge values (the value at the centre), r1 the slope.
    """
    z = 0.0 + 0.0j
    hh = 0.0
    for i, det in enumerate(ev.detectors):
        he = physics.detector_strain(het.edges, theta, det, ev.gmst)
        r = he / het.h0_edges[i]
        width = het.edges[1:] - het.edges[:-1]
        r0 = 0.5 * (r[:-1] + r[1:])
        r1 = (r[1:] - r[:-1]) / width
        z += complex(np.sum(het.A0[i] * r0 + het.A1[i] * r1))
        hh += float(np.sum(het.B0[i] * np.abs(r0) ** 2 + 2.0 * het.B1[i] * np.real(r0 * np.conj(r1))))
    return z, hh


def het_loglike(ev: Event, het: Het, theta):
    """Heterodyned logL: r = h/h0 linear in each bin, r0 at the centre, r1 slope.

    <d|h> ~ Re sum_b (A0 r0 + A1 r1),  <h|h> ~ sum_b (B0 |r0|^2 + 2 B1 Re(r0 r1*)).
    The phase-marginalised form uses the complex Z = sum_b (A0 r0 + A1 r1).
    -1/2 <d|d> is the same constant as in the full likelihood.
    """
    theta = np.asarray(theta, dtype=np.float64).copy()
    if ev.phase_marginalised:
        theta[IDX["phic"]] = 0.0
    z, hh = het_overlap(ev, het, theta)
    dd = sum(inner_product(d, d, s, ev.df) for d, s in zip(ev.data, ev.psds))
    if ev.phase_marginalised:
        x = abs(z)
        return x + math.log(i0e(x)) - 0.5 * hh - 0.5 * dd
    return z.real - 0.5 * hh - 0.5 * dd


# --------------------------------------------------------------------------
# Time marginalisation (Sec. 3.1 and App. A): t_c summed over a grid of time
# shifts, on the heterodyned bins (the direct sum) and, as its full-resolution
# analogue, on the whole frequency grid.
# --------------------------------------------------------------------------
def time_grid(params, n_nodes):
    """Midpoint nodes of the uniform t_c prior [lo, hi]:
    t_j = lo + (j + 1/2) (hi - lo) / N_t, each carrying prior mass 1 / N_t."""
    p = params[IDX["tc"]]
    if p.kind != PRIOR_UNIFORM:
        raise ValueError("time marginalisation needs a uniform t_c prior")
    return p.lo + (np.arange(n_nodes) + 0.5) * ((p.hi - p.lo) / n_nodes)


def _node_log_weight(ev: Event, z):
    """The t_c-dependent part of logL at one node: log I0(|Z|) with phi_c
    marginalised, Re Z otherwise."""
    if ev.phase_marginalised:
        x = np.abs(z)
        return x + np.log(i0e(x))
    return np.real(z)


def het_time_overlaps(ev: Event, het: Het, theta, t_nodes):
    """Z(t_j): the heterodyned overlap of the template moved to t_c = t_j, for
    every node; and <h|h>, which a time shift leaves unchanged, taken once
    with t_c at the fiducial's value."""
    theta = np.asarray(theta, dtype=np.float64).copy()
    if ev.phase_marginalised:
        theta[IDX["phic"]] = 0.0
    theta[IDX["tc"]] = het.theta_fid[IDX["tc"]]
    _, hh = het_overlap(ev, het, theta)
    z = np.empty(len(t_nodes), dtype=np.complex128)
    for j, t in enumerate(t_nodes):
        theta[IDX["tc"]] = t
        z[j] = het_overlap(ev, het, theta)[0]
    return z, hh


def het_time_log_weights(ev: Event, het: Het, theta, n_nodes):
    """log of the conditional weights of t_c on its grid (up to a constant)."""
    z, _ = het_time_overlaps(ev, het, theta, time_grid(ev.params, n_nodes))
    return _node_log_weight(ev, z)


def het_loglike_time_marg(ev: Event, het: Het, theta, n_nodes):
    """Heterodyned logL with t_c marginalised over its uniform prior:
    log( (1/N_t) sum_j exp(logL_het(theta, t_c = t_j)) ), <h|h> at the
    fiducial's t_c (the theta[tc] passed in is ignored)."""
    t = time_grid(ev.params, n_nodes)
    z, hh = het_time_overlaps(ev, het, theta, t)
    ell = _node_log_weight(ev, z)
    m = float(np.max(ell))
    dd = sum(inner_product(d, d, s, ev.df) for d, s in zip(ev.data, ev.psds))
    return m + math.log(float(np.sum(np.exp(ell - m)))) - math.log(n_nodes) - 0.5 * hh - 0.5 * dd


def full_time_overlaps(ev: Event, theta, t_nodes):
    """Full-grid Z(t_j) = sum_i 4 df sum_f d_i* h_i(t_c = t_j) / S_i and <h|h>."""
    theta = np.asarray(theta, dtype=np.float64).copy()
    if ev.phase_marginalised:
        theta[IDX["phic"]] = 0.0
    z = np.empty(len(t_nodes), dtype=np.complex128)
    hh = None
    for j, t in enumerate(t_nodes):
        theta[IDX["tc"]] = t
        hs = strains(ev, theta)
        z[j] = sum(complex_overlap(d, h, s, ev.df) for d, h, s in zip(ev.data, hs, ev.psds))
        if hh is None:
            hh = sum(inner_product(h, h, s, ev.df) for h, s in zip(hs, ev.psds))
    return z, hh


def loglike_time_marg_full(ev: Event, theta, n_nodes):
    """Full-resolution logL with t_c marginalised on the same midpoint grid."""
    t = time_grid(ev.params, n_nodes)
    z, hh = full_time_overlaps(ev, theta, t)
    ell = _node_log_weight(ev, z)
    m = float(np.max(ell))
    dd = sum(inner_product(d, d, s, ev.df) for d, s in zip(ev.data, ev.psds))
    return m + math.log(float(np.sum(np.exp(ell - m)))) - math.log(n_nodes) - 0.5 * hh - 0.5 * dd


def draw_time_node(log_w, q):
    """Index of the grid node drawn by the uniform q from weights exp(log_w):
    the first node whose cumulative weight reaches q times the total."""
    w = np.exp(np.asarray(log_w, dtype=np.float64) - np.max(log_w))
    c = np.cumsum(w)
    return int(min(np.searchsorted(c, q * c[-1], side="left"), len(c) - 1))
