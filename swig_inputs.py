"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the inference method itself: it draws the
random numbers, states the noise model (a closed-form design-like PSD), the
detector site table, the frequency grid and the sidereal-time reference.  The
waveform, the detector projection, the inner products, the likelihood and the
sampler live elsewhere (the oracle for the CPU reference, the CUDA library for
the product), and each side computes them independently.

Workloads follow the injection study of Sec. 4.1 and Table I of the paper
(128 s segment, 20-2048 Hz, H1/L1/V1 network, reference GPS 1187008882) with
the substitutions a closed-form PSD forces (Bilby PSD files are not shipped).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Speed of light (exact, SI) and the mean Earth radius of the spherical-Earth
# site model.
C_SI = 299792458.0
EARTH_RADIUS_M = 6.371e6

# Parameter slots of the 13-vector used throughout (Table I of the paper, with
# aligned spins chi1, chi2 standing in for the spin-sphere triples).
PARAM_NAMES = ("mc", "q", "chi1", "chi2", "lambda1", "lambda2", "dl", "iota",
               "psi", "ra", "dec", "tc", "phic")
N_PARAMS = len(PARAM_NAMES)
IDX = {n: i for i, n in enumerate(PARAM_NAMES)}

# Prior kinds (inverse-CDF families) and parameter modes.
PRIOR_UNIFORM, PRIOR_SINE, PRIOR_COSINE, PRIOR_POWER2 = 0, 1, 2, 3
MODE_SAMPLE, MODE_FIXED, MODE_MARG = 0, 1, 2


def frequency_grid(f_min: float, f_max: float, df: float) -> np.ndarray:
    """Bins k*df for k = ceil(f_min/df) .. floor(f_max/df), both ends inclusive."""
    k0 = int(math.ceil(f_min / df - 1e-9))
    k1 = int(math.floor(f_max / df + 1e-9))
    return np.arange(k0, k1 + 1, dtype=np.float64) * df


def design_psd(f: np.ndarray, scale: float = 1.0) -> np.ndarray:
    """Closed-form aLIGO-like one-sided PSD [1/Hz].

    Ajith (2011), PRD 84, 084037: analytic fit to the zero-detuned high-power
    Advanced LIGO noise curve, S(f) = 1e-49 [x^-4.14 - 5 x^-2 + 111 (1 - x^2 +
    x^4/2) / (1 + x^2/2)], x = f / 215 Hz.  ``scale`` multiplies the PSD (4.0
    gives the Virgo-like curve used for V1: amplitude spectral density x2).
    """
    x = np.asarray(f, dtype=np.float64) / 215.0
    s = x**-4.14 - 5.0 * x**-2 + 111.0 * (1.0 - x**2 + 0.5 * x**4) / (1.0 + 0.5 * x**2)
    return scale * 1e-49 * s


# Approximate public site values: geodetic latitude and longitude [deg], and
# the azimuths of the x and y arms [deg, clockwise from local north].
SITES = {
    "H1": (46.455, -119.408, 324.0, 234.0),
    "L1": (30.563, -90.774, 252.3, 162.3),
    "V1": (43.631, 10.504, 19.4, 289.4),
}
PSD_SCALE = {"H1": 1.0, "L1": 1.0, "V1": 4.0}


def site_vectors(name: str):
    """Vertex [m] and unit arm vectors (Earth-fixed frame) on a spherical Earth."""
    lat, lon, az_x, az_y = (math.radians(v) for v in SITES[name])
    up = np.array([math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), math.sin(lat)])
    east = np.array([-math.sin(lon), math.cos(lon), 0.0])
    north = np.array([-math.sin(lat) * math.cos(lon), -math.sin(lat) * math.sin(lon), math.cos(lat)])
    arm = lambda az: math.cos(az) * north + math.sin(az) * east
    return EARTH_RADIUS_M * up, arm(az_x), arm(az_y)


def gmst_from_gps(gps: float) -> float:
    """Greenwich mean sidereal time [rad] at a GPS time (18 leap seconds).

    Uses the common linear approximation GMST[h] = 18.697374558 +
    24.06570982441908 D, D = days from J2000.0 (UT1 taken equal to UTC).
    The value is only a shared convention fixing Earth's orientation.
    """
    jd = 2444244.5 + (gps - 18.0) / 86400.0
    hours = 18.697374558 + 24.06570982441908 * (jd - 2451545.0)
    return (hours % 24.0) / 24.0 * 2.0 * math.pi


REFERENCE_GPS = 1187008882.0


def colored_noise(rng: np.random.Generator, psd: np.ndarray, df: float) -> np.ndarray:
    """Complex Gaussian noise with Re, Im ~ N(0, S/(4 df)) independently."""
    sigma = np.sqrt(psd / (4.0 * df))
    return sigma * (rng.standard_normal(psd.shape) + 1j * rng.standard_normal(psd.shape))


@dataclass
class Param:
    """One slot of the 13-vector: prior family, bounds, mode and Gibbs block."""
    kind: int
    lo: float
    hi: float
    mode: int = MODE_SAMPLE
    value: float = 0.0       # used when mode == MODE_FIXED
    block: int = 0


@dataclass
class Workload:
    """A synthetic event: grid, detectors, PSDs, injection, prior and sampler knobs."""
    name: str
    f_min: float
    f_max: float
    df: float
    detectors: tuple
    params: list
    injection: np.ndarray        # 13-vector: physical values, or unit-cube values if inj_unit
    target_snr: float
    noise_seed: int
    sampler_seed: int
    nlive: int
    nrep: int                    # chains (k deletions per iteration)
    steps_per_dim: int
    sweeps: int = 1
    het_bins: int = 0
    inj_unit: bool = False       # injection holds unit-cube coordinates of every slot
    freqs: np.ndarray = field(default=None, repr=False)

    def __post_init__(self):
        self.freqs = frequency_grid(self.f_min, self.f_max, self.df)

    @property
    def n_bins(self) -> int:
        return int(self.freqs.size)

    def psds(self):
        return [design_psd(self.freqs, PSD_SCALE[d]) for d in self.detectors]

    def noise(self):
        rng = np.random.default_rng(self.noise_seed)
        return [colored_noise(rng, s, self.df) for s in self.psds()]

    def sampled(self):
        return [i for i, p in enumerate(self.params) if p.mode == MODE_SAMPLE]


def _bns_params(block_sky=True):
    """Table I ranges (aligned-spin, tidal), Gibbs blocks following Sec. 3.2."""
    P = Param
    return [
        P(PRIOR_UNIFORM, 1.5, 2.5, block=0),            # mc
        P(PRIOR_UNIFORM, 0.5, 1.0, block=0),            # q
        P(PRIOR_UNIFORM, -0.05, 0.05, block=1),         # chi1
        P(PRIOR_UNIFORM, -0.05, 0.05, block=2),         # chi2
        P(PRIOR_UNIFORM, 0.0, 5000.0, block=0),         # lambda1
        P(PRIOR_UNIFORM, 0.0, 5000.0, block=0),         # lambda2
        P(PRIOR_POWER2, 30.0, 150.0, block=7),          # dl
        P(PRIOR_SINE, 0.0, math.pi, block=3),           # iota
        P(PRIOR_UNIFORM, 0.0, math.pi, block=5),        # psi
        P(PRIOR_UNIFORM, 0.0, 2 * math.pi, block=4),    # ra
        P(PRIOR_COSINE, -math.pi / 2, math.pi / 2, block=4),  # dec
        P(PRIOR_UNIFORM, -0.1, 0.1, block=6),           # tc
        P(PRIOR_UNIFORM, 0.0, 2 * math.pi, mode=MODE_MARG, block=8),  # phic
    ]


def unit_to_prior_draw(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform draws on the unit cube (mapped to parameters by each side)."""
    return rng.random((n, N_PARAMS))


def config1(nlive: int = 100) -> Workload:
    """One H1-like detector, 4 s, 20-1024 Hz, df = 0.25 Hz, FP64, 4 free params.

    Gibbs blocks {Mc, q, t_c} and {d_L}: the chirp mass and the coalescence
    time are strongly correlated on this short segment, and a joint block lets
    the covariance-directed slice move along that ridge (a separate t_c block
    mixed it much more slowly)."""
    P = Param
    params = [
        P(PRIOR_UNIFORM, 1.1, 1.3, block=0),
        P(PRIOR_UNIFORM, 0.5, 1.0, block=0),
        P(PRIOR_UNIFORM, 0, 0, MODE_FIXED, 0.0),
        P(PRIOR_UNIFORM, 0, 0, MODE_FIXED, 0.0),
        P(PRIOR_UNIFORM, 0, 0, MODE_FIXED, 0.0),
        P(PRIOR_UNIFORM, 0, 0, MODE_FIXED, 0.0),
        P(PRIOR_UNIFORM, 20.0, 200.0, block=1),
        P(PRIOR_UNIFORM, 0, 0, MODE_FIXED, 0.4),
        P(PRIOR_UNIFORM, 0, 0, MODE_FIXED, 0.3),
        P(PRIOR_UNIFORM, 0, 0, MODE_FIXED, 1.2),
        P(PRIOR_UNIFORM, 0, 0, MODE_FIXED, 0.5),
        P(PRIOR_UNIFORM, -0.1, 0.1, block=0),
        P(PRIOR_UNIFORM, 0, 0, MODE_FIXED, 0.0),
    ]
    inj = np.array([1.2, 0.8, 0, 0, 0, 0, 100.0, 0.4, 0.3, 1.2, 0.5, 0.0, 0.0])
    return Workload("cfg1_h1_4s", 20.0, 1024.0, 0.25, ("H1",), params, inj, 20.0,
                    noise_seed=2000, sampler_seed=3000, nlive=nlive, nrep=max(1, nlive // 10),
                    steps_per_dim=5)


def config2(nlive: int = 1000, seed_index: int = 0) -> Workload:
    """H1/L1/V1, 128 s, 20-2048 Hz, df = 1/128 Hz, 13 params, network SNR 25."""
    params = _bns_params()
    rng = np.random.default_rng(1000 + seed_index)
    u = rng.random(N_PARAMS)
    # Injection drawn from the prior's unit cube; each side maps u -> theta
    # with its own prior transform, then rescales d_L to the target SNR.
    return Workload("cfg2_hlv_128s", 20.0, 2048.0, 1.0 / 128.0, ("H1", "L1", "V1"), params,
                    u, 25.0, noise_seed=2000 + seed_index, sampler_seed=3000 + seed_index,
                    nlive=nlive, nrep=nlive // 10, steps_per_dim=5, inj_unit=True)
