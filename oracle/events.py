"""Oracle-side synthesis of an event from a seeded workload description.

Data d_i = h_i(theta_inj) + n_i with the oracle's own waveform and projection;
the noise and every other random draw come from ``swig_inputs``.  The CUDA
path receives the arrays built here through its C-ABI in the parity tests.
"""
from __future__ import annotations

import numpy as np

from swig_inputs import IDX, MODE_FIXED, REFERENCE_GPS, Workload, gmst_from_gps, site_vectors
from . import physics
from .likelihood import Event, optimal_snr_sq


def injection_theta(wl: Workload):
    """Physical 13-vector of the injection with d_L set for the target SNR."""
    if wl.inj_unit:
        theta = np.zeros(13)
        for i, p in enumerate(wl.params):
            if p.mode == MODE_FIXED:
                theta[i] = p.value
            else:
                theta[i] = physics.prior_transform_1d(wl.injection[i], p.kind, p.lo, p.hi)
    else:
        theta = np.array(wl.injection, dtype=np.float64)
    return theta


def build_event(wl: Workload, zero_noise=False, rescale_snr=True):
    freqs = wl.freqs
    dets = [physics.Detector(*site_vectors(n)) for n in wl.detectors]
    psds = wl.psds()
    gmst = gmst_from_gps(REFERENCE_GPS)
    theta = injection_theta(wl)
    ev = Event(freqs, wl.df, [np.zeros(freqs.size, complex)] * len(dets), psds, dets, gmst, wl.params)
    if rescale_snr and wl.target_snr > 0:
        snr = np.sqrt(optimal_snr_sq(ev, theta))
        theta[IDX["dl"]] *= snr / wl.target_snr
    hs = [physics.detector_strain(freqs, theta, d, gmst) for d in dets]
    if zero_noise:
        data = hs
    else:
        data = [h + n for h, n in zip(hs, wl.noise())]
    ev.data = data
    return ev, theta
