"""Pins of the oracle's forward model against closed forms and textbook series."""
import math

import numpy as np
import pytest

import swig_inputs as si
from oracle import physics


def test_psd_positive_and_low_frequency_wall():
    f = np.linspace(10.0, 4096.0, 20000)
    s = si.design_psd(f)
    assert np.all(s > 0)
    # Ajith (2011) fit: S(f)/1e-49 -> x^-4.14 dominates at low frequency
    x = 5.0 / 215.0
    assert si.design_psd(np.array([5.0]))[0] / 1e-49 == pytest.approx(x**-4.14 - 5 * x**-2, rel=1e-4)
    # bucket minimum near 215 Hz * O(1)
    assert 100.0 < f[np.argmin(s)] < 400.0


def test_grid_counts():
    assert si.frequency_grid(20, 1024, 0.25).size == 4017
    assert si.frequency_grid(20, 2048, 1 / 128).size == 259585


def test_detector_tensor_traceless_symmetric():
    for name in si.SITES:
        r, x, y = si.site_vectors(name)
        D = physics.detector_tensor(x, y)
        assert abs(np.trace(D)) < 1e-15
        assert np.allclose(D, D.T)
        assert abs(np.dot(x, y)) < 1e-12 and abs(np.linalg.norm(r) - si.EARTH_RADIUS_M) < 1e-6


def _detector_frame_angles(x, y, n):
    z = np.cross(x, y)
    cth = float(np.dot(n, z))
    phi = math.atan2(float(np.dot(n, y)), float(np.dot(n, x)))
    return cth, phi


def test_antenna_power_matches_textbook_L_shape():
    # F+^2 + Fx^2 = (1+cos^2 th)^2 cos^2(2 ph) / 4 + cos^2 th sin^2(2 ph)
    # for a source at polar angle th, azimuth ph in the frame (x arm, y arm, x cross y)
    rng = np.random.default_rng(0)
    for name in si.SITES:
        r, x, y = si.site_vectors(name)
        D = physics.detector_tensor(x, y)
        for _ in range(50):
            ra, dec, psi, g = rng.uniform(0, 2 * np.pi), np.arcsin(rng.uniform(-1, 1)), rng.uniform(0, np.pi), rng.uniform(0, 2 * np.pi)
            fp, fx = physics.antenna_patterns(D, ra, dec, psi, g)
            cth, ph = _detector_frame_angles(x, y, physics.source_direction(ra, dec, g))
            expect = 0.25 * (1 + cth**2) ** 2 * math.cos(2 * ph) ** 2 + cth**2 * math.sin(2 * ph) ** 2
            assert fp**2 + fx**2 == pytest.approx(expect, rel=1e-12, abs=1e-14)
            # invariance under psi and the bound <= 1
            fp2, fx2 = physics.antenna_patterns(D, ra, dec, psi + 0.7, g)
            assert fp2**2 + fx2**2 == pytest.approx(fp**2 + fx**2, rel=1e-12, abs=1e-14)
            assert fp**2 + fx**2 <= 1 + 1e-12


def test_time_delays():
    rH, _, _ = si.site_vectors("H1")
    rL, _, _ = si.site_vectors("L1")
    bound = np.linalg.norm(rH - rL) / si.C_SI
    assert 0.0095 < bound < 0.0102          # ~10 ms light travel time H1-L1
    g = 0.3
    rng = np.random.default_rng(1)
    for _ in range(200):
        ra, dec = rng.uniform(0, 2 * np.pi), np.arcsin(rng.uniform(-1, 1))
        d = physics.time_delay(rH, ra, dec, g) - physics.time_delay(rL, ra, dec, g)
        assert abs(d) <= bound * (1 + 1e-12)
    # source along the baseline saturates the bound; overhead source arrives R/c early
    b = (rL - rH) / np.linalg.norm(rL - rH)
    dec = math.asin(b[2]); ra = math.atan2(b[1], b[0]) + g
    d = physics.time_delay(rH, ra, dec, g) - physics.time_delay(rL, ra, dec, g)
    assert d == pytest.approx(bound, rel=1e-9)
    u = rH / np.linalg.norm(rH)
    assert physics.time_delay(rH, math.atan2(u[1], u[0]) + g, math.asin(u[2]), g) == pytest.approx(-si.EARTH_RADIUS_M / si.C_SI, rel=1e-12)


def _chirp_time_series(v, eta, beta=0.0, sigma=0.0):
    """tau(v) = t_c - t(f): Blanchet, Living Rev. Rel. 17 (2014) 2, the 3.5PN
    time-to-coalescence series in x = v^2 (non-spinning), with the 1.5PN
    spin-orbit (8/5) beta v^3 and 2PN spin-spin -2 sigma v^4 corrections of
    Poisson & Will (1995) / Cutler & Flanagan (1994)."""
    pi, g = math.pi, physics.EULER_GAMMA
    c = (1.0
         + (743.0 / 252.0 + 11.0 / 3.0 * eta) * v**2
         + (-32.0 / 5.0 * pi + 8.0 / 5.0 * beta) * v**3
         + (3058673.0 / 508032.0 + 5429.0 / 504.0 * eta + 617.0 / 72.0 * eta**2 - 2.0 * sigma) * v**4
         - pi * (7729.0 / 252.0 - 13.0 / 3.0 * eta) * v**5
         + (-10052469856691.0 / 23471078400.0 + 128.0 / 3.0 * pi**2 + 6848.0 / 105.0 * g
            + (3147553127.0 / 3048192.0 - 451.0 / 12.0 * pi**2) * eta
            - 15211.0 / 1728.0 * eta**2 + 25565.0 / 1296.0 * eta**3
            + 3424.0 / 105.0 * np.log(16.0 * v**2)) * v**6
         + pi * (-15419335.0 / 127008.0 - 75703.0 / 756.0 * eta + 14809.0 / 378.0 * eta**2) * v**7)
    return c


@pytest.mark.parametrize("mc,q,chi1,chi2", [(1.2, 0.8, 0.0, 0.0), (2.0, 0.55, 0.04, -0.03), (1.6, 1.0, -0.05, 0.05)])
def test_spa_time_frequency_relation(mc, q, chi1, chi2):
    """(1/2 pi) dPsi_int/df = -tau(f) with the textbook chirp-time series.

    The Newtonian term is the quadrupole chirp time (5/256) Mc (pi Mc f)^(-8/3)
    = 5 M / (256 eta v^8); the bracket is Blanchet's series, independent of
    the alpha_k list being tested.  Central finite differences in FP64.
    """
    eta = physics.symmetric_mass_ratio(q)
    m_s = physics.total_mass_seconds(mc, q)
    m1, m2 = 1 / (1 + q), q / (1 + q)
    beta = (113 / 12 * m1**2 + 25 / 4 * eta) * chi1 + (113 / 12 * m2**2 + 25 / 4 * eta) * chi2
    sigma = 79 / 8 * eta * chi1 * chi2
    f = np.array([20.0, 35.0, 60.0, 120.0, 300.0])
    h = 1e-3
    psi = lambda ff: physics.taylorf2_phase_intrinsic(ff, mc, q, chi1, chi2, 0.0, 0.0)
    dpsi = (psi(f + h) - psi(f - h)) / (2 * h) / (2 * math.pi)
    v = np.cbrt(math.pi * m_s * f)
    tau = 5.0 * m_s / (256.0 * eta * v**8) * _chirp_time_series(v, eta, beta, sigma)
    newt = 5.0 / 256.0 * mc * physics.MTSUN_S * (math.pi * mc * physics.MTSUN_S * f) ** (-8.0 / 3.0)
    assert np.allclose(5.0 * m_s / (256.0 * eta * v**8), newt, rtol=1e-12, atol=0)
    assert np.allclose(dpsi, -tau, rtol=2e-8, atol=0)


def test_newtonian_only_phase_is_quadrupole_chirp():
    mc, q = 1.4, 0.9
    f = np.array([25.0, 50.0, 100.0])
    h = 1e-3
    psi = lambda ff: physics.taylorf2_phase_intrinsic(ff, mc, q, 0, 0, 0, 0, orders={0})
    dpsi = (psi(f + h) - psi(f - h)) / (2 * h) / (2 * math.pi)
    mcs = mc * physics.MTSUN_S
    assert np.allclose(dpsi, -5.0 / 256.0 * mcs * (math.pi * mcs * f) ** (-8.0 / 3.0), rtol=1e-8, atol=0)


def test_tidal_lambda_tilde():
    # equal masses and equal Lambda: Lambda~ = Lambda, dLambda~ = 0
    for lam in (0.0, 400.0, 5000.0):
        assert physics.tidal_lambda_tilde(0.25, 0.0, lam, lam) == pytest.approx(lam, rel=1e-14, abs=1e-12)
        assert physics.tidal_delta_lambda_tilde(0.25, 0.0, lam, lam) == pytest.approx(0.0, abs=1e-12)
    # Favata (2014) form: Lambda~ = 16/13 [(m1 + 12 m2) m1^4 L1 + (m2 + 12 m1) m2^4 L2] / M^5
    rng = np.random.default_rng(2)
    for _ in range(50):
        q = rng.uniform(0.3, 1.0); l1, l2 = rng.uniform(0, 5000, 2)
        m1, m2 = 1 / (1 + q), q / (1 + q)
        eta = physics.symmetric_mass_ratio(q)
        fav = 16.0 / 13.0 * ((m1 + 12 * m2) * m1**4 * l1 + (m2 + 12 * m1) * m2**4 * l2)
        assert physics.tidal_lambda_tilde(eta, m1 - m2, l1, l2) == pytest.approx(fav, rel=1e-12)
        # label swap: Lambda~ symmetric, dLambda~ antisymmetric
        assert physics.tidal_lambda_tilde(eta, m2 - m1, l2, l1) == pytest.approx(fav, rel=1e-12)
        a = physics.tidal_delta_lambda_tilde(eta, m1 - m2, l1, l2)
        b = physics.tidal_delta_lambda_tilde(eta, m2 - m1, l2, l1)
        assert a == pytest.approx(-b, rel=1e-12, abs=1e-9)


def test_tidal_phase_terms_enter_as_stated():
    """alpha10 = -(39/2) Lambda~ gives the 5PN tidal chirp-time term (39/2) Lambda~ v^10."""
    mc, q, lam = 1.8, 1.0, 3000.0
    eta = 0.25
    m_s = physics.total_mass_seconds(mc, q)
    f = np.array([100.0, 400.0])
    h = 1e-3
    dpsi = lambda o: ((physics.taylorf2_phase_intrinsic(f + h, mc, q, 0, 0, lam, lam, orders=o)
                       - physics.taylorf2_phase_intrinsic(f - h, mc, q, 0, 0, lam, lam, orders=o)) / (2 * h) / (2 * math.pi))
    v = np.cbrt(math.pi * m_s * f)
    lead = 5.0 * m_s / (256.0 * eta * v**8)
    assert np.allclose(dpsi({10}), -lead * (39.0 / 2.0) * lam * v**10, rtol=1e-7, atol=0)


def test_prior_transforms_invert_cdf():
    u = np.linspace(0.001, 0.999, 101)
    x = physics.prior_transform_1d(u, si.PRIOR_SINE, 0.0, math.pi)
    assert np.allclose((1 - np.cos(x)) / 2, u, atol=1e-13)
    x = physics.prior_transform_1d(u, si.PRIOR_COSINE, -math.pi / 2, math.pi / 2)
    assert np.allclose((np.sin(x) + 1) / 2, u, atol=1e-13)
    x = physics.prior_transform_1d(u, si.PRIOR_POWER2, 30.0, 150.0)
    assert np.allclose((x**3 - 30.0**3) / (150.0**3 - 30.0**3), u, atol=1e-13)
    x = physics.prior_transform_1d(u, si.PRIOR_UNIFORM, -0.1, 0.1)
    assert np.allclose((x + 0.1) / 0.2, u, atol=1e-14)


def test_polarization_amplitudes():
    """|h+| / |hx| = (1 + cos^2 i) / (2 |cos i|); hx leads h+ by a quarter cycle."""
    f = np.array([30.0, 200.0])
    th = np.array([1.5, 0.9, 0, 0, 0, 0, 100.0, 0.7, 0.2, 1.0, 0.3, 0.01, 0.5])
    hp, hx = physics.polarizations(f, th)
    c = math.cos(0.7)
    assert np.allclose(np.abs(hp) / np.abs(hx), (1 + c * c) / (2 * abs(c)))
    assert np.allclose(hx / hp, -1j * c / (0.5 * (1 + c * c)))
    # Newtonian amplitude: |h+| at iota=0 equals A f^-7/6
    th[7] = 0.0
    hp, _ = physics.polarizations(f, th)
    assert np.allclose(np.abs(hp), physics.amplitude_prefactor(1.5, 100.0) * f ** (-7 / 6), rtol=1e-12, atol=0)


def test_amplitude_is_the_spa_of_the_quadrupole_chirp():
    """Face-on, h+(t) = h0 cos Phi(t) with the quadrupole amplitude
    h0 = 4 (c / d) (G Mc / c^3)^(5/3) (pi f)^(2/3) and chirp rate
    df/dt = (96/5) pi^(8/3) (G Mc / c^3)^(5/3) f^(11/3).  The stationary-phase
    transform gives |h+~(f)| = (h0 / 2) (df/dt)^(-1/2), which must equal
    A f^(-7/6)."""
    f = np.array([20.0, 87.0, 400.0, 1500.0])
    for mc, d in ((1.2, 40.0), (2.3, 150.0)):
        m = mc * physics.MTSUN_S
        h0 = 4.0 * (physics.C_SI / (d * physics.MPC_M)) * m ** (5.0 / 3.0) * (math.pi * f) ** (2.0 / 3.0)
        fdot = 96.0 / 5.0 * math.pi ** (8.0 / 3.0) * m ** (5.0 / 3.0) * f ** (11.0 / 3.0)
        spa = 0.5 * h0 / np.sqrt(fdot)
        assert np.allclose(physics.amplitude_prefactor(mc, d) * f ** (-7.0 / 6.0), spa, rtol=1e-12, atol=0)


def test_prior_transforms_on_sub_ranges():
    """The inverse CDFs on ranges other than the Table I ones: the prior mass
    below x(u), by adaptive quadrature of the unnormalised density, is u."""
    from scipy import integrate
    u = np.array([0.02, 0.3, 0.5, 0.77, 0.98])
    cases = ((si.PRIOR_SINE, 0.3, 2.0, math.sin), (si.PRIOR_COSINE, -0.4, 1.1, math.cos),
             (si.PRIOR_POWER2, 10.0, 40.0, lambda x: x * x), (si.PRIOR_UNIFORM, -3.0, 5.0, lambda x: 1.0))
    for kind, lo, hi, dens in cases:
        x = physics.prior_transform_1d(u, kind, lo, hi)
        total = integrate.quad(dens, lo, hi, epsabs=0, epsrel=1e-13)[0]
        mass = np.array([integrate.quad(dens, lo, xi, epsabs=0, epsrel=1e-13)[0] for xi in x]) / total
        assert np.allclose(mass, u, atol=1e-11), kind


@pytest.mark.parametrize("q,lam1,lam2", [(1.0, 400.0, 400.0), (0.7, 300.0, 900.0), (0.5, 50.0, 2000.0), (0.9, 1000.0, 10.0)])
def test_tidal_terms_equal_the_per_body_form(q, lam1, lam2):
    """The 5PN and 6PN tidal coefficients written per body (Vines, Flanagan &
    Hinderer 2011): with X_A = m_A / M and X_B = 1 - X_A,
      alpha_10 = -sum_A (24 / X_A) (1 + 11 X_B) X_A^5 Lambda_A,
      alpha_12 = -sum_A 5 / (28 X_A) (3179 - 919 X_A - 2286 X_A^2 + 260 X_A^3) X_A^5 Lambda_A.
    The Lambda-tilde / delta-Lambda-tilde form must reproduce both for unequal
    masses and deformabilities (this fixes delta-Lambda-tilde's coefficients
    and the sign of its 6PN term, which vanish at equal masses)."""
    a = physics.pn_phase_coefficients(1.3, q, 0.0, 0.0, lam1, lam2)
    m1, m2 = 1.0 / (1.0 + q), q / (1.0 + q)
    a10 = a12 = 0.0
    for xa, xb, lam in ((m1, m2, lam1), (m2, m1, lam2)):
        a10 -= 24.0 / xa * (1.0 + 11.0 * xb) * xa**5 * lam
        a12 -= 5.0 / (28.0 * xa) * (3179.0 - 919.0 * xa - 2286.0 * xa**2 + 260.0 * xa**3) * xa**5 * lam
    assert a[10] == pytest.approx(a10, rel=1e-12, abs=0)
    assert a[12] == pytest.approx(a12, rel=1e-12, abs=0)


@pytest.mark.parametrize("q,chi1,chi2", [(0.55, 0.04, -0.03), (0.8, -0.05, -0.02), (0.93, 0.05, 0.05), (1.0, 0.03, -0.01)])
def test_spin_terms_against_independent_forms(q, chi1, chi2):
    """The aligned-spin parts of alpha_3 and alpha_4, against two published
    forms written in other variables (so a wrong 113/12, 25/4, 79/8 or a swapped
    mass weight fails):

    * 1.5PN spin-orbit in the symmetric/antisymmetric spins chi_s = (chi1 +
      chi2)/2, chi_a = (chi1 - chi2)/2, delta = (m1 - m2)/M, as Ajith (2011,
      PRD 84, 084037) writes the non-precessing TaylorF2 phase:
      alpha_3 spin part = (113/3)(chi_s + delta chi_a) - (76/3) eta chi_s;
    * 2PN spin-spin from Kidder (1995, PRD 52, 821):
      sigma = eta/48 [721 (L.chi1)(L.chi2) - 247 chi1.chi2], which for spins
      along L is eta (721 - 247)/48 chi1 chi2; alpha_4 spin part = -10 sigma.
    """
    mc = 1.7
    eta = physics.symmetric_mass_ratio(q)
    m1, m2 = 1 / (1 + q), q / (1 + q)
    delta = m1 - m2
    a_spin = physics.pn_phase_coefficients(mc, q, chi1, chi2, 0.0, 0.0)
    a_zero = physics.pn_phase_coefficients(mc, q, 0.0, 0.0, 0.0, 0.0)
    chi_s, chi_a = 0.5 * (chi1 + chi2), 0.5 * (chi1 - chi2)
    so = 113.0 / 3.0 * (chi_s + delta * chi_a) - 76.0 / 3.0 * eta * chi_s
    assert a_spin[3] - a_zero[3] == pytest.approx(so, rel=1e-12, abs=1e-15)
    sigma = eta / 48.0 * (721.0 * chi1 * chi2 - 247.0 * chi1 * chi2)
    assert a_spin[4] - a_zero[4] == pytest.approx(-10.0 * sigma, rel=1e-12, abs=1e-15)
    # the other orders do not see the spins
    for k in (0, 2, 5, 6, 7):
        assert a_spin[k] == a_zero[k]
