"""Forward model in FP64: prior transform, TaylorF2 waveform, detector response.

Follows Sec. 3.1 of the paper (templates h_i(theta) projected onto a detector
network) with the aligned-spin, tidal TaylorF2 model that stands in for the
paper's IMRPhenomPv2_NRTidalv2 (which needs ripple-level model code).

Conventions (shared with the CUDA path by definition, not by code):
  * Fourier transform h~(f) = int h(t) exp(-2 pi i f t) dt.
  * h+~ = (1 + cos^2 i)/2 * A f^(-7/6) exp(-i Psi),  hx~ = -i cos i * A f^(-7/6) exp(-i Psi)
    with Psi(f) = 2 pi f t_c - phi_c + Psi_int(f).
  * Detector i sees h_i~ = (F+ h+~ + Fx hx~) exp(-2 pi i f dt_i), dt_i = -n.r_i / c.
  * Polarisation basis X = -cos(psi) e_east + sin(psi) e_north,
    Y = sin(psi) e_east + cos(psi) e_north on the sky at the source direction n.
"""
from __future__ import annotations

import math

import numpy as np

from swig_inputs import (C_SI, IDX, MODE_FIXED, MODE_MARG, N_PARAMS, PRIOR_COSINE, PRIOR_POWER2,
                         PRIOR_SINE, PRIOR_UNIFORM)

EULER_GAMMA = 0.57721566490153286061
# G M_sun / c^3 [s] from the IAU 2015 (Resolution B3) nominal solar mass
# parameter G M_sun = 1.3271244e20 m^3 s^-2, and the parsec-based Mpc [m].
GM_SUN_SI = 1.3271244e20
MTSUN_S = GM_SUN_SI / C_SI**3
MPC_M = 3.0856775814913673e22


# --------------------------------------------------------------------------
# Prior transform (Table I): unit hypercube -> physical parameters
# --------------------------------------------------------------------------
def prior_transform_1d(u, kind, lo, hi):
    """Inverse CDF of one Table I prior family on [lo, hi]."""
    u = np.asarray(u, dtype=np.float64)
    if kind == PRIOR_UNIFORM:
        return lo + u * (hi - lo)
    if kind == PRIOR_SINE:          # p(x) ~ sin x
        return np.arccos(np.cos(lo) - u * (np.cos(lo) - np.cos(hi)))
    if kind == PRIOR_COSINE:        # p(x) ~ cos x
        return np.arcsin(np.sin(lo) + u * (np.sin(hi) - np.sin(lo)))
    if kind == PRIOR_POWER2:        # p(x) ~ x^2
        return np.cbrt(lo**3 + u * (hi**3 - lo**3))
    raise ValueError(f"unknown prior kind {kind}")


def detector_frame(vertex_a, vertex_b):
    """Orthonormal frame of the baseline from detector b to detector a:
    ez along the baseline, ex the Earth's rotation axis made orthogonal to ez,
    ey = ez x ex (Earth-fixed coordinates)."""
    ez = np.asarray(vertex_a, dtype=np.float64) - np.asarray(vertex_b, dtype=np.float64)
    ez = ez / np.linalg.norm(ez)
    pole = np.array([0.0, 0.0, 1.0])
    ex = pole - ez * (pole @ ez)
    if np.linalg.norm(ex) < 1e-12:
        axis = np.array([1.0, 0.0, 0.0])
        ex = axis - ez * (axis @ ez)
    ex = ex / np.linalg.norm(ex)
    return ex, np.cross(ez, ex), ez


def frame_to_radec(az, zen, frame, gmst):
    """(azimuth, zenith) about ez of `frame` -> (RA, Dec) at sidereal time gmst."""
    ex, ey, ez = frame
    n = math.sin(zen) * math.cos(az) * ex + math.sin(zen) * math.sin(az) * ey + math.cos(zen) * ez
    dec = math.asin(max(-1.0, min(1.0, float(n[2]))))
    ra = (math.atan2(float(n[1]), float(n[0])) + gmst) % (2.0 * math.pi)
    return ra, dec


def prior_transform(u_sampled, params, sky=None):
    """Map the sampled unit-cube coordinates to the full 13-vector theta.

    ``u_sampled`` has one column per parameter with mode SAMPLE, in slot order.
    Fixed slots take their value; marginalised slots are set to 0.  With
    ``sky = (frame, gmst)`` slots 9 and 10 are sampled as (azimuth, zenith)
    about the frame's ez and converted to (RA, Dec).
    """
    u_sampled = np.atleast_2d(np.asarray(u_sampled, dtype=np.float64))
    theta = np.zeros((u_sampled.shape[0], N_PARAMS))
    j = 0
    for i, p in enumerate(params):
        if p.mode == MODE_FIXED:
            theta[:, i] = p.value
        elif p.mode == MODE_MARG:
            theta[:, i] = 0.0
        else:
            theta[:, i] = prior_transform_1d(u_sampled[:, j], p.kind, p.lo, p.hi)
            j += 1
    if sky is not None:
        frame, gmst = sky
        for r in range(theta.shape[0]):
            theta[r, IDX["ra"]], theta[r, IDX["dec"]] = frame_to_radec(theta[r, IDX["ra"]], theta[r, IDX["dec"]],
                                                                       frame, gmst)
    return theta


# --------------------------------------------------------------------------
# TaylorF2 (aligned spin, tidal), Newtonian amplitude
# --------------------------------------------------------------------------
def symmetric_mass_ratio(q):
    return q / (1.0 + q) ** 2


def total_mass_seconds(mc, q):
    """Total mass G M / c^3 [s] from chirp mass [Msun] and q = m2/m1 <= 1."""
    return mc * symmetric_mass_ratio(q) ** (-0.6) * MTSUN_S


def tidal_lambda_tilde(eta, delta, lam1, lam2):
    """Wade et al. 2014 (PRD 89, 103012), Eq. 5: effective tidal parameter.

    ``delta`` = (m1 - m2) / M, signed (sqrt(1 - 4 eta) when m1 >= m2).
    """
    return (8.0 / 13.0) * ((1 + 7 * eta - 31 * eta**2) * (lam1 + lam2)
                           + delta * (1 + 9 * eta - 11 * eta**2) * (lam1 - lam2))


def tidal_delta_lambda_tilde(eta, delta, lam1, lam2):
    """Wade et al. 2014, Eq. 6: second tidal combination entering at 6PN."""
    return 0.5 * (delta * (1 - 13272.0 / 1319 * eta + 8944.0 / 1319 * eta**2) * (lam1 + lam2)
                  + (1 - 15910.0 / 1319 * eta + 32850.0 / 1319 * eta**2
                     + 3380.0 / 1319 * eta**3) * (lam1 - lam2))


def pn_phase_coefficients(mc, q, chi1, chi2, lam1, lam2, orders=None):
    """PN coefficients alpha_k of Psi = 3/(128 eta v^5) sum_k alpha_k v^k.

    Non-spinning terms: Buonanno, Iyer, Ochsner, Pan & Sathyaprakash 2009
    (PRD 80, 084043), Eq. 3.18.  Aligned spin: 1.5PN spin-orbit beta and 2PN
    spin-spin sigma (Poisson & Will 1995; Cutler & Flanagan 1994).  Tides:
    5PN and 6PN terms of Wade et al. 2014, Eq. 4.  Returned as a dict with the
    v-independent parts; alpha5 and alpha6 also carry log-v parts returned as
    'alpha5_log' (multiplies ln(v / v_lso)) and 'alpha6_log' (multiplies ln 4v).
    ``orders`` (set of ints) keeps only the listed v-powers, for the pins.
    """
    eta = symmetric_mass_ratio(q)
    m1 = 1.0 / (1.0 + q)
    m2 = q / (1.0 + q)
    delta = math.sqrt(max(1.0 - 4.0 * eta, 0.0))
    beta = (113.0 / 12.0 * m1**2 + 25.0 / 4.0 * eta) * chi1 + (113.0 / 12.0 * m2**2 + 25.0 / 4.0 * eta) * chi2
    sigma = 79.0 / 8.0 * eta * chi1 * chi2
    pi = math.pi
    a = {
        0: 1.0,
        1: 0.0,
        2: 3715.0 / 756.0 + 55.0 / 9.0 * eta,
        3: -16.0 * pi + 4.0 * beta,
        4: 15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta**2 - 10.0 * sigma,
        5: pi * (38645.0 / 756.0 - 65.0 / 9.0 * eta),
        6: (11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi**2 - 6848.0 / 21.0 * EULER_GAMMA
            + (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi**2) * eta
            + 76055.0 / 1728.0 * eta**2 - 127825.0 / 1296.0 * eta**3),
        7: pi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta**2),
    }
    lt = tidal_lambda_tilde(eta, delta, lam1, lam2)
    dlt = tidal_delta_lambda_tilde(eta, delta, lam1, lam2)
    a[10] = -39.0 / 2.0 * lt
    a[12] = -3115.0 / 64.0 * lt + 6595.0 / 364.0 * delta * dlt
    a["alpha5_log"] = 3.0 * a[5]
    a["alpha6_log"] = -6848.0 / 21.0
    if orders is not None:
        for k in list(a.keys()):
            base = 5 if k == "alpha5_log" else 6 if k == "alpha6_log" else k
            if base not in orders:
                a[k] = 0.0
    return a


V_LSO = 1.0 / math.sqrt(6.0)


def taylorf2_phase_intrinsic(f, mc, q, chi1, chi2, lam1, lam2, orders=None):
    """Psi_int(f) [rad] = -pi/4 + 3/(128 eta v^5) [sum_k alpha_k v^k + logs].

    v = (pi M f)^(1/3).  The full phase is Psi = 2 pi f t_c - phi_c + Psi_int.
    """
    f = np.asarray(f, dtype=np.float64)
    eta = symmetric_mass_ratio(q)
    m_s = total_mass_seconds(mc, q)
    v = np.cbrt(math.pi * m_s * f)
    a = pn_phase_coefficients(mc, q, chi1, chi2, lam1, lam2, orders)
    series = np.zeros_like(v)
    for k in (0, 1, 2, 3, 4, 5, 6, 7, 10, 12):
        series += a[k] * v**k
    series += a["alpha5_log"] * np.log(v / V_LSO) * v**5
    series += a["alpha6_log"] * np.log(4.0 * v) * v**6
    const = -math.pi / 4.0 if orders is None else 0.0
    return const + 3.0 / (128.0 * eta * v**5) * series


def amplitude_prefactor(mc, dl_mpc):
    """A = sqrt(5/24) pi^(-2/3) (c / d_L) (G Mc / c^3)^(5/6)  [s^(1/6)]."""
    mc_s = mc * MTSUN_S
    return math.sqrt(5.0 / 24.0) * math.pi ** (-2.0 / 3.0) * mc_s ** (5.0 / 6.0) / (dl_mpc * MPC_M / C_SI)


def polarizations(f, theta):
    """Geocentric h+~, hx~ at the bins f for one 13-vector theta."""
    mc, q, chi1, chi2, lam1, lam2, dl, iota, psi, ra, dec, tc, phic = theta
    psi_int = taylorf2_phase_intrinsic(f, mc, q, chi1, chi2, lam1, lam2)
    phase = 2.0 * math.pi * f * tc - phic + psi_int
    core = amplitude_prefactor(mc, dl) * f ** (-7.0 / 6.0) * np.exp(-1j * phase)
    ci = math.cos(iota)
    return 0.5 * (1.0 + ci * ci) * core, -1j * ci * core


# --------------------------------------------------------------------------
# Detector response
# --------------------------------------------------------------------------
def detector_tensor(x_arm, y_arm):
    """D = (x x^T - y y^T) / 2 for unit arm vectors."""
    x = np.asarray(x_arm, dtype=np.float64)
    y = np.asarray(y_arm, dtype=np.float64)
    return 0.5 * (np.outer(x, x) - np.outer(y, y))


def source_direction(ra, dec, gmst):
    """Unit vector from Earth's centre to the source (Earth-fixed frame)."""
    lon = ra - gmst
    return np.array([math.cos(dec) * math.cos(lon), math.cos(dec) * math.sin(lon), math.sin(dec)])


def polarization_basis(ra, dec, psi, gmst):
    lon = ra - gmst
    e_east = np.array([-math.sin(lon), math.cos(lon), 0.0])
    e_north = np.array([-math.sin(dec) * math.cos(lon), -math.sin(dec) * math.sin(lon), math.cos(dec)])
    X = -math.cos(psi) * e_east + math.sin(psi) * e_north
    Y = math.sin(psi) * e_east + math.cos(psi) * e_north
    return X, Y


def antenna_patterns(D, ra, dec, psi, gmst):
    """F+ = D:(XX - YY), Fx = D:(XY + YX)."""
    X, Y = polarization_basis(ra, dec, psi, gmst)
    e_plus = np.outer(X, X) - np.outer(Y, Y)
    e_cross = np.outer(X, Y) + np.outer(Y, X)
    return float(np.sum(D * e_plus)), float(np.sum(D * e_cross))


def time_delay(vertex_m, ra, dec, gmst):
    """Arrival time at the detector minus arrival time at Earth's centre [s]."""
    return -float(np.dot(source_direction(ra, dec, gmst), vertex_m)) / C_SI


class Detector:
    def __init__(self, vertex_m, x_arm, y_arm):
        self.vertex = np.asarray(vertex_m, dtype=np.float64)
        self.D = detector_tensor(x_arm, y_arm)


def detector_strain(f, theta, det: Detector, gmst):
    """h_i~(f) = (F+ h+~ + Fx hx~) exp(-2 pi i f dt_i)."""
    ra, dec, psi = theta[IDX["ra"]], theta[IDX["dec"]], theta[IDX["psi"]]
    fp, fx = antenna_patterns(det.D, ra, dec, psi, gmst)
    dt = time_delay(det.vertex, ra, dec, gmst)
    hp, hx = polarizations(f, theta)
    return (fp * hp + fx * hx) * np.exp(-2j * math.pi * f * dt)
