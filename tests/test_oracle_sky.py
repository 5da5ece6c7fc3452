"""Pins of the detector-frame sky parameterisation in the oracle: the frame
is orthonormal and right-handed, zenith 0 points along the baseline, the map
to (RA, Dec) is a rotation (angles preserved), and an isotropic prior in the
frame is isotropic in (RA, Dec)."""
import math

import numpy as np
from scipy import stats

import swig_inputs as si
from oracle import physics

GMST = si.gmst_from_gps(si.REFERENCE_GPS)


def _frame():
    va, _, _ = si.site_vectors("H1")
    vb, _, _ = si.site_vectors("L1")
    return physics.detector_frame(va, vb), va, vb


def test_frame_orthonormal_right_handed():
    (ex, ey, ez), va, vb = _frame()
    for a in (ex, ey, ez):
        assert abs(np.linalg.norm(a) - 1.0) < 1e-14
    assert abs(ex @ ey) < 1e-14 and abs(ey @ ez) < 1e-14 and abs(ex @ ez) < 1e-14
    assert np.allclose(np.cross(ex, ey), ez, atol=1e-14)
    assert np.allclose(ez, (va - vb) / np.linalg.norm(va - vb), atol=1e-15)


def test_zenith_zero_is_the_baseline_direction():
    frame, va, vb = _frame()
    for az in (0.0, 1.0, 4.0):
        ra, dec = physics.frame_to_radec(az, 0.0, frame, GMST)
        assert np.allclose(physics.source_direction(ra, dec, GMST), frame[2], atol=1e-12)


def test_azimuth_runs_from_ex_towards_ey():
    """On the equator of the frame (zenith pi/2) azimuth 0 is ex and pi/2 is
    ey, so with the right-handed frame the azimuth turns about ez."""
    frame, _, _ = _frame()
    for az, axis in ((0.0, frame[0]), (0.5 * math.pi, frame[1]), (math.pi, -frame[0])):
        ra, dec = physics.frame_to_radec(az, 0.5 * math.pi, frame, GMST)
        assert np.allclose(physics.source_direction(ra, dec, GMST), axis, atol=1e-12)


def test_map_preserves_angles():
    frame, _, _ = _frame()
    rng = np.random.default_rng(1)
    for _ in range(20):
        a1, a2 = rng.random(2) * 2 * math.pi
        z1, z2 = np.arccos(1 - 2 * rng.random(2))
        n1 = np.array([math.sin(z1) * math.cos(a1), math.sin(z1) * math.sin(a1), math.cos(z1)])
        n2 = np.array([math.sin(z2) * math.cos(a2), math.sin(z2) * math.sin(a2), math.cos(z2)])
        r1 = physics.source_direction(*physics.frame_to_radec(a1, z1, frame, GMST), GMST)
        r2 = physics.source_direction(*physics.frame_to_radec(a2, z2, frame, GMST), GMST)
        assert abs(n1 @ n2 - r1 @ r2) < 1e-12


def test_isotropic_prior_stays_isotropic():
    frame, _, _ = _frame()
    rng = np.random.default_rng(2)
    params = [si.Param(si.PRIOR_UNIFORM, 0, 0, si.MODE_FIXED, 0.0) for _ in range(si.N_PARAMS)]
    params[si.IDX["ra"]] = si.Param(si.PRIOR_UNIFORM, 0.0, 2 * math.pi)
    params[si.IDX["dec"]] = si.Param(si.PRIOR_SINE, 0.0, math.pi)
    th = physics.prior_transform(rng.random((20000, 2)), params, sky=(frame, GMST))
    sd = np.sin(th[:, si.IDX["dec"]])
    ra = th[:, si.IDX["ra"]]
    assert stats.kstest((sd + 1) / 2, "uniform").pvalue > 1e-3
    assert stats.kstest(ra / (2 * math.pi), "uniform").pvalue > 1e-3
