"""The library's host-side preparation, checked on the CPU (no GPU needed):
`host_harness.cu` compiles the C-ABI source into a small program that calls
the pure host routines, and their results must equal the oracle's and
numpy's.

* heterodyne bin edges (Sec. 3.4): the grid indices of the equal-dephasing
  and geometric rules, bit for bit against the oracle (integer work), on the
  4 s and 128 s grids;
* the Gauss-Legendre rule of the distance marginal against numpy's leggauss;
* the detector sky frame against the oracle's detector_frame.
"""
import ctypes
import json
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import swig_inputs as si
from oracle import likelihood as L
from oracle import physics

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    from paper_2607_28265_gb300 import build, swig
    if not os.path.exists(swig.LIB_PATH):
        build.build()
    lib_dir = os.path.dirname(swig.LIB_PATH)
    exe = str(tmp_path_factory.mktemp("host") / "host_harness")
    cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2607_28265_gb300", "csrc"),
           os.path.join(ROOT, "tests", "host_harness.cu"), "-o", exe, "-L", lib_dir, "-lswig",
           "-Xlinker", "-rpath", "-Xlinker", lib_dir]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def _run(exe, *args):
    r = subprocess.run([exe] + [str(a) for a in args], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (args, r.returncode, r.stderr)
    return json.loads(r.stdout)


@pytest.mark.parametrize("which,bins", [("cfg1", (10, 150, 300, 451, 600, 1000)), ("cfg2", (1000, 5000))])
def test_het_edge_indices_equal_the_oracle(harness, which, bins):
    wl = si.config1() if which == "cfg1" else si.config2()
    freqs = wl.freqs
    for nb in bins:
        for spacing in (0, 1):
            out = _run(harness, "edges", repr(wl.f_min), repr(wl.f_max), repr(wl.df), nb, spacing)
            assert out["n_bins"] == freqs.size and out["k_min"] * wl.df == freqs[0]
            _, want = (L.phase_bound_edges(freqs, nb) if spacing == 0 else L.geometric_edges(freqs, nb))
            assert np.array_equal(out["idx"], want), (which, nb, spacing)


@pytest.mark.parametrize("n", [8, 64])
def test_gauss_legendre_rule(harness, n):
    """Against the roots of P_n and the weights 2 / ((1 - x^2) P_n'(x)^2) in
    40-digit arithmetic (mpmath, Newton from numpy's estimates), and against
    numpy's leggauss (itself good to ~1e-12 relative in the weights at n = 64)."""
    mpmath = pytest.importorskip("mpmath")
    out = _run(harness, "gl", n)
    xn, wn = np.polynomial.legendre.leggauss(n)
    with mpmath.workdps(40):
        xr, wr = [], []
        for x0 in xn:
            x = mpmath.mpf(float(x0))
            for _ in range(60):
                dp = n * (x * mpmath.legendre(n, x) - mpmath.legendre(n - 1, x)) / (x * x - 1)
                x -= mpmath.legendre(n, x) / dp
            dp = n * (x * mpmath.legendre(n, x) - mpmath.legendre(n - 1, x)) / (x * x - 1)
            xr.append(float(x))
            wr.append(float(2 / ((1 - x * x) * dp * dp)))
    assert np.allclose(out["x"], xr, rtol=0, atol=4e-16)
    assert np.allclose(out["w"], wr, rtol=3e-13, atol=0)
    assert np.allclose(out["w"], wn, rtol=5e-12, atol=0)
    assert abs(sum(out["w"]) - 2.0) < 1e-13


def test_sky_frame_equals_the_oracle(harness):
    gmst = si.gmst_from_gps(si.REFERENCE_GPS)
    for a, b in (("H1", "L1"), ("L1", "V1"), ("V1", "H1")):
        va, _, _ = si.site_vectors(a)
        vb, _, _ = si.site_vectors(b)
        out = _run(harness, "frame", *[repr(float(v)) for v in va], *[repr(float(v)) for v in vb], repr(gmst))
        ex, ey, ez = physics.detector_frame(va, vb)
        assert np.allclose(out["ex"], ex, rtol=0, atol=1e-14)
        assert np.allclose(out["ey"], ey, rtol=0, atol=1e-14)
        assert np.allclose(out["ez"], ez, rtol=0, atol=1e-14)


# The phase basis P(f) = sum_j c_j phi_j(f) of the mixed path, in the
# library's order: f^-5/3, f^-1, f^-2/3, f^-1/3, ln f, f^1/3, f^1/3 ln f,
# f^2/3, f^5/3, f^7/3, 1 (power, carries ln f).
_BASIS = [(-5 / 3, 0), (-1.0, 0), (-2 / 3, 0), (-1 / 3, 0), (0.0, 1), (1 / 3, 0), (1 / 3, 1), (2 / 3, 0),
          (5 / 3, 0), (7 / 3, 0), (0.0, 0)]


def _falling(p, n):
    out = 1.0
    for i in range(n):
        out *= p - i
    return out


def _deriv(p, lg, n, f):
    """n-th derivative of f^p (ln f)^lg, by the Leibniz rule with
    d^k ln f = (-1)^(k-1) (k-1)! f^-k."""
    f = np.asarray(f, dtype=np.float64)
    if not lg:
        return _falling(p, n) * f ** (p - n)
    s = sum(math.comb(n, k) * _falling(p, n - k) * (-1) ** (k - 1) * math.factorial(k - 1) for k in range(1, n + 1))
    return f ** (p - n) * (_falling(p, n) * np.log(f) + s)


@pytest.mark.parametrize("which", ["cfg1", "cfg2"])
def test_tile_plan_meets_its_remainder_bound(harness, which):
    """The tiles of the mixed-precision phase: they cover the grid in powers of
    two (2048 at most, aligned to 32-bin chunks), their stored basis values are
    the analytic derivatives, and over every tile the degree-6 Taylor
    remainder, summed over the basis with the coefficient bounds of the prior
    box, stays below 1e-8 cycles."""
    wl = si.config1() if which == "cfg1" else si.config2()
    out = _run(harness, "tiles", repr(wl.f_min), repr(wl.f_max), repr(wl.df))
    tiles, cmax = out["tiles"], np.array(out["cmax"])
    n = wl.freqs.size
    k = 0
    for i, t in enumerate(tiles):
        assert t["k0"] == k
        span = 1 << max(0, (t["nbins"] - 1).bit_length())
        assert span <= 2048 and t["inv_T"] == 1.0 / span
        if i < len(tiles) - 1:
            assert t["nbins"] == span
        assert t["k0"] % min(span, 32) == 0
        k += t["nbins"]
    assert k == n
    worst = 0.0
    for t in tiles:
        fa = (out["k_min"] + t["k0"]) * wl.df
        x = np.arange(t["nbins"], dtype=np.float64)
        f = fa + x * wl.df
        span = 1.0 / t["inv_T"]
        r = 0.0
        for j, (p, lg) in enumerate(_BASIS):
            if p == 0.0 and not lg:
                continue
            d = [float(_deriv(p, lg, m, fa)) for m in range(7)]
            assert t["val"][j] == pytest.approx(d[0], rel=1e-14, abs=0)
            assert t["slope"][j] == pytest.approx(d[1] * wl.df, rel=1e-14, abs=0)
            for m in range(5):
                want = d[m + 2] * (wl.df * span) ** (m + 2) / math.factorial(m + 2)
                assert t["poly"][m][j] == pytest.approx(want, rel=2e-7, abs=1e-300)
            taylor = sum(d[m] * (x * wl.df) ** m / math.factorial(m) for m in range(7))
            exact = _deriv(p, lg, 0, f)
            r += cmax[j] * float(np.max(np.abs(exact - taylor)))
        worst = max(worst, r)
    assert worst < 1e-8, worst


@pytest.mark.parametrize("theta", [(1.2, 0.8, 0.0, 0.0, 0.0, 0.0), (1.5, 0.5, 0.05, -0.05, 0.0, 5000.0),
                                   (2.5, 1.0, -0.05, 0.05, 5000.0, 0.0), (1.87, 0.71, 0.013, -0.037, 812.0, 2240.0)])
def test_phase_coefficients_equal_the_oracle_phase(harness, theta):
    """The TaylorF2 phase in cycles, sum_j c_j(theta) phi_j(f) with the
    coefficients of the set-up code the device also runs, equals the oracle's
    Psi_int(f) / 2 pi over 20-2048 Hz (h ~ exp(-2 pi i (P(f) + f tau)))."""
    mc, q, chi1, chi2, lam1, lam2 = theta
    c = np.array(_run(harness, "coeffs", *[repr(float(v)) for v in theta])["c"])
    f = np.geomspace(20.0, 2048.0, 3001)
    P = sum(c[j] * _deriv(p, lg, 0, f) for j, (p, lg) in enumerate(_BASIS))
    want = physics.taylorf2_phase_intrinsic(f, mc, q, chi1, chi2, lam1, lam2) / (2 * math.pi)
    assert np.allclose(P, want, rtol=1e-12, atol=1e-9)


def test_amplitude_equals_the_oracle(harness):
    for mc in (0.9, 1.2, 1.87, 2.9):
        got = _run(harness, "amp", repr(mc))["amp"]
        assert got == pytest.approx(physics.amplitude_prefactor(mc, 1.0), rel=1e-14, abs=0)


def test_log_bessel_i0_forms(harness):
    """log I0 (FP64, both branches and their seam at x = 20) against scipy's
    i0e: within 2e-14 relative, and 1e-12 absolute just past the seam, where the
    asymptotic series' truncation (~3e-13) is largest.  The FP32
    log(I0(x) e^-x) of the mixed epilogues within 2e-6: FP32 summation of the
    power series below x = 20, ~1e-6 there."""
    from scipy.special import i0e
    xs = [0.0, 1e-3, 0.5, 5.0, 19.99, 20.01, 25.0, 100.0, 700.0, 5000.0]
    out = _run(harness, "logi0", *[repr(x) for x in xs])
    want = np.log(i0e(xs))
    assert np.allclose(out["log_i0"], want + np.array(xs), rtol=2e-14, atol=1e-12)
    assert np.allclose(out["log_i0e_f32"], want, rtol=0, atol=2e-6)


@pytest.mark.parametrize("kind,lo,hi", [(si.PRIOR_POWER2, 30.0, 150.0), (si.PRIOR_UNIFORM, 20.0, 200.0)])
@pytest.mark.parametrize("phase_marg", [0, 1])
def test_distance_marginal_epilogue_equals_the_oracle(harness, kind, lo, hi, phase_marg):
    """The 64-node distance marginal of the epilogues (template at 1 Mpc: Z1,
    H1) against the oracle's adaptive quadrature, from no signal to a peak
    inside, at and beyond the prior edges; tolerance as on the GPU."""
    p = si.Param(kind, lo, hi, si.MODE_MARG)
    dd = 4.0e3
    for snr2_at_100, d_peak in ((0.0, 100.0), (50.0, 80.0), (400.0, 100.0), (900.0, 35.0), (600.0, 140.0),
                                (400.0, 20.0), (400.0, 400.0), (3.0, 60.0)):
        h1 = snr2_at_100 * 100.0 ** 2
        z1 = complex(h1 / d_peak, 0.3 * h1 / d_peak) if phase_marg else complex(h1 / d_peak, 0.0)
        got = _run(harness, "distmarg", kind, repr(lo), repr(hi), phase_marg, repr(z1.real), repr(z1.imag),
                   repr(h1), repr(dd))["logl"]
        want = L.log_distance_integral(z1, h1, dd, p, bool(phase_marg))
        assert abs(got - want) <= 1e-6 * abs(want) + 1e-4, (snr2_at_100, d_peak, got, want)


def test_prior_inverse_cdfs_equal_the_oracle(harness):
    u = [0.0, 0.013, 0.25, 0.5, 0.77, 0.999, 1.0]
    for kind, lo, hi in ((si.PRIOR_UNIFORM, -0.1, 0.1), (si.PRIOR_SINE, 0.0, math.pi), (si.PRIOR_SINE, 0.3, 2.0),
                         (si.PRIOR_COSINE, -math.pi / 2, math.pi / 2), (si.PRIOR_COSINE, -0.4, 1.1),
                         (si.PRIOR_POWER2, 30.0, 150.0)):
        got = _run(harness, "prior", kind, repr(lo), repr(hi), *[repr(x) for x in u])["x"]
        want = physics.prior_transform_1d(np.array(u), kind, lo, hi)
        assert np.allclose(got, want, rtol=1e-13, atol=1e-14), kind


def test_sky_frame_map_equals_the_oracle(harness):
    gmst = si.gmst_from_gps(si.REFERENCE_GPS)
    va, _, _ = si.site_vectors("H1")
    vb, _, _ = si.site_vectors("L1")
    frame = physics.detector_frame(va, vb)
    rng = np.random.default_rng(4)
    for az, zen in zip(rng.random(6) * 2 * math.pi, np.arccos(1 - 2 * rng.random(6))):
        got = _run(harness, "sky", *[repr(float(v)) for v in va], *[repr(float(v)) for v in vb], repr(gmst),
                   repr(float(az)), repr(float(zen)))
        ra, dec = physics.frame_to_radec(az, zen, frame, gmst)
        assert abs(got["dec"] - dec) < 1e-12
        assert abs(math.remainder(got["ra"] - ra, 2 * math.pi)) < 1e-12


def test_prior_map_places_sampled_and_fixed_slots_like_the_oracle(harness):
    """The full 13-slot map of the sampler and the batched transform (sampled
    coordinates in slot order, fixed slots at their values) against the
    oracle's prior_transform, on the 128 s and 4 s workloads' priors."""
    rng = np.random.default_rng(6)
    for wl in (si.config2(), si.config1()):
        params = wl.params
        spec = "\n".join(f"{p.kind} {p.mode} {p.lo!r} {p.hi!r} {p.value!r}" for p in params)
        u = rng.random((5, len(wl.sampled())))
        rows = "\n".join(" ".join(repr(float(v)) for v in r) for r in u)
        r = subprocess.run([harness, "priormap"], input=spec + "\n" + rows + "\n", capture_output=True, text=True,
                           timeout=60)
        assert r.returncode == 0, r.stderr
        got = np.array(json.loads(r.stdout)["theta"])
        want = physics.prior_transform(u, params)
        keep = [i for i, p in enumerate(params) if p.mode != si.MODE_MARG]
        assert got.shape == want.shape
        assert np.allclose(got[:, keep], want[:, keep], rtol=1e-13, atol=1e-14)


def test_binding_structs_match_the_c_abi(harness):
    """The ctypes structures of the Python binding have the C structs' field
    order, offsets and sizes (compiled from include/swig.h), and every field
    the header declares."""
    from paper_2607_28265_gb300 import swig
    out = _run(harness, "abi")
    for cname, py in (("swig_param", swig.SwigParam), ("swig_sampler_cfg", swig.SwigSamplerCfg),
                      ("swig_result", swig.SwigResult)):
        c = out[cname]
        assert c["size"] == ctypes.sizeof(py), cname
        assert [f for f, _ in c["fields"]] == [f[0] for f in py._fields_], cname
        for f, off in c["fields"]:
            assert getattr(py, f).offset == off, (cname, f)


def test_time_marginalisation_tables_equal_the_hat_weights(harness):
    """The library's edge weights g_ie and per-step rotations from the
    oracle's summary data: g_ie is the coefficient of r_i(e) in the per-bin
    overlap (the linear-in-bin ratio's hat functions), w_e = exp(-2 pi i f_e dt);
    FP32 storage."""
    wl = si.config2()
    from oracle import events
    ev, th = events.build_event(wl)
    het = L.het_setup(ev, th, 300)
    nb, nd, dt = het.edges.size - 1, len(ev.detectors), 0.2 / 2000
    a01 = np.concatenate([np.stack([het.A0[i].real, het.A0[i].imag, het.A1[i].real, het.A1[i].imag], axis=1).ravel()
                          for i in range(nd)])
    text = f"{nb} {nd} {dt!r}\n" + " ".join(repr(float(x)) for x in het.edges) + "\n" + \
        " ".join(repr(float(x)) for x in a01) + "\n"
    r = subprocess.run([harness, "tmtables"], input=text, capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    out = json.loads(r.stdout)
    g = np.array(out["g"]).reshape(nd, nb + 1, 2)
    w = np.array(out["w"]).reshape(nb + 1, 2)
    # coefficient of r(e) in sum_b A0 (r_b + r_b+1)/2 + A1 (r_b+1 - r_b)/width_b, by unit vectors
    width = het.edges[1:] - het.edges[:-1]
    for i in range(nd):
        for e in (0, 1, nb // 2, nb - 1, nb):
            r_unit = np.zeros(nb + 1)
            r_unit[e] = 1.0
            want = np.sum(het.A0[i] * 0.5 * (r_unit[:-1] + r_unit[1:]) + het.A1[i] * (r_unit[1:] - r_unit[:-1]) / width)
            scale = np.max(np.abs(het.A0[i]))
            assert abs(complex(*g[i, e]) - want) <= 1e-6 * scale, (i, e)
    want_w = np.exp(-2j * math.pi * het.edges * dt)
    assert np.allclose(w[:, 0] + 1j * w[:, 1], want_w, rtol=0, atol=2e-7)


def test_heterodyne_summary_data_equal_the_oracle(harness):
    """The library's summary data (compensated FP64 sums) from the oracle's own
    fiducial waveform, data and PSDs against the oracle's het_setup: A0, A1
    to 1e-12 of each detector's largest |A0|, |A1|; B0, B1 to FP32 storage."""
    from oracle import events
    wl = si.config1()
    ev, th = events.build_event(wl)
    het = L.het_setup(ev, th, 300)
    _, idx = L.phase_bound_edges(ev.freqs, 300)
    nb, n = idx.size - 1, ev.freqs.size
    h0 = L.strains(ev, th)
    parts = [f"{n} {nb} {len(ev.detectors)} {ev.df!r}", " ".join(repr(float(x)) for x in ev.freqs),
             " ".join(str(int(k)) for k in idx)]
    for d, s, h in zip(ev.data, ev.psds, h0):
        parts.append(" ".join(repr(float(x)) for x in np.stack([d.real, d.imag], axis=1).ravel()))
        parts.append(" ".join(repr(float(x)) for x in s))
        parts.append(" ".join(repr(float(x)) for x in np.stack([h.real, h.imag], axis=1).ravel()))
    r = subprocess.run([harness, "hetsum"], input="\n".join(parts) + "\n", capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    out = json.loads(r.stdout)
    a01 = np.array(out["a01"]).reshape(len(ev.detectors), nb, 4)
    b01 = np.array(out["b01"]).reshape(len(ev.detectors), nb, 2)
    for i in range(len(ev.detectors)):
        A0 = a01[i, :, 0] + 1j * a01[i, :, 1]
        A1 = a01[i, :, 2] + 1j * a01[i, :, 3]
        assert np.max(np.abs(A0 - het.A0[i])) <= 1e-12 * np.max(np.abs(het.A0[i]))
        assert np.max(np.abs(A1 - het.A1[i])) <= 1e-12 * np.max(np.abs(het.A1[i]))
        assert np.allclose(b01[i, :, 0], het.B0[i], rtol=1e-7, atol=0)
        assert np.max(np.abs(b01[i, :, 1] - het.B1[i])) <= 1e-7 * np.max(np.abs(het.B1[i]))


def test_full_grid_data_weights_equal_the_inner_products(harness):
    """The weighted data of the full-grid likelihood against the oracle's
    inner products: K_i = <f^-7/6 | f^-7/6>_i, <d|d> summed over detectors,
    D_i(f) = 4 df conj(d_i) f^-7/6 / S_i at sampled bins, max |D_i|."""
    from oracle import events
    wl = si.config2()
    ev, _ = events.build_event(wl)
    stride = 997
    text = []
    for d, s in zip(ev.data, ev.psds):
        text.append(" ".join(repr(float(x)) for x in np.stack([d.real, d.imag], axis=1).ravel()))
        text.append(" ".join(repr(float(x)) for x in s))
    r = subprocess.run([harness, "weights", repr(wl.f_min), repr(wl.f_max), repr(wl.df), str(len(ev.data)), str(stride)],
                       input="\n".join(text) + "\n", capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    out = json.loads(r.stdout)
    f = ev.freqs
    amp = f ** (-7.0 / 6.0)
    dd = sum(L.inner_product(d, d, s, ev.df) for d, s in zip(ev.data, ev.psds))
    assert out["dd"] == pytest.approx(dd, rel=1e-12, abs=0)
    D = np.concatenate([4.0 * ev.df * np.conj(d) * amp / s for d, s in zip(ev.data, ev.psds)])
    for i, s in enumerate(ev.psds):
        assert out["K"][i] == pytest.approx(L.inner_product(amp, amp, s, ev.df), rel=1e-12, abs=0)
        Di = D[i * f.size:(i + 1) * f.size]
        assert out["dmax"][i] == pytest.approx(np.max(np.abs(Di)), rel=1e-14, abs=0)
    sample = D[::stride]
    assert np.allclose(np.array(out["dre"]) + 1j * np.array(out["dim"]), sample, rtol=1e-14, atol=0)


@pytest.mark.parametrize("n_t", [64, 1000, 2000, 4096])
def test_time_pass_nufft_tables_reproduce_the_direct_sum(harness, n_t):
    """The tables of the non-uniform FFT time pass (het_nufft_tables): gather
    lists of the kernel-weighted edge values, 1 / Phi per node.  Applied in
    FP64 here (gather, an inverse FFT with exponent +2 pi i, deconvolution)
    they give Z(dt_j) = sum_e y_e exp(-2 pi i f_e dt_j) on the uniform node grid
    to ~1e-8 of sum |y_e| (the kernel's error for width 8 at twofold
    oversampling), on the 128 s grid's 5,000-bin equal-phase edges, for node
    spacings below 1 / (2 f_max)."""
    wl = si.config2()
    f = np.arange(int(np.ceil(wl.f_min / wl.df)), int(np.floor(wl.f_max / wl.df)) + 1) * wl.df
    edges, _ = L.phase_bound_edges(f, 5000)
    dt = 0.2 / n_t
    inp = f"{len(edges)} " + " ".join(repr(float(x)) for x in edges)
    r = subprocess.run([harness, "nufft", str(n_t), repr(dt)], input=inp, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout)
    M, j0 = d["M"], d["j0"]
    if n_t == 64:
        # nodes 3.1 ms apart: f_e dt wraps past one cycle, a grid point's edges
        # are no longer consecutive, and the tables are declined (direct sum)
        assert M == 0 and d["ptr"] == []
        return
    assert M >= 2 * n_t and M & (M - 1) == 0 and j0 == n_t // 2
    ptr, edge, wt, corr = (np.array(d[k]) for k in ("ptr", "edge", "wt", "corr"))
    assert len(ptr) == M + 1 and len(edge) == M  # first edge per grid point (its edges are consecutive)
    rng = np.random.default_rng(n_t)
    y = rng.normal(size=len(edges)) + 1j * rng.normal(size=len(edges))
    t0 = -0.1 + 0.5 * dt
    c = y * np.exp(-2j * np.pi * edges * (t0 + j0 * dt))
    b = np.array([np.sum(wt[ptr[l]:ptr[l + 1]] * c[edge[l]:edge[l] + ptr[l + 1] - ptr[l]]) for l in range(M)])
    X = np.fft.ifft(b) * M
    j = np.arange(n_t)
    Z = X[(j - j0) % M] * corr
    Zd = np.exp(-2j * np.pi * np.outer(t0 + j * dt, edges)) @ y
    assert np.max(np.abs(Z - Zd)) < 1e-7 * np.sum(np.abs(y))


# Basis of the phase in cycles, phi_j(f) (the order of the device's Basis enum):
# f^-5/3, f^-1, f^-2/3, f^-1/3, ln f, f^1/3, f^1/3 ln f, f^2/3, f^5/3, f^7/3, 1.
_BASIS_POW = (-5 / 3, -1.0, -2 / 3, -1 / 3, 0.0, 1 / 3, 1 / 3, 2 / 3, 5 / 3, 7 / 3, 0.0)
_BASIS_LOG = (0, 0, 0, 0, 1, 0, 1, 0, 0, 0, 0)


def _basis(f):
    f = np.asarray(f, dtype=np.float64)
    out = []
    for p, lg in zip(_BASIS_POW, _BASIS_LOG):
        v = f ** p if p != 0.0 else np.ones_like(f)
        out.append(v * np.log(f) if lg else v)
    return np.array(out)  # [NBASIS][n]


@pytest.mark.parametrize("which,nb,spacing", [("cfg2", 5000, 0), ("cfg1", 450, 1), ("cfg1", 300, 0)])
def test_het_chunk_taylor_form_within_its_remainder_bound(harness, which, nb, spacing):
    """The heterodyned contraction's chunk tables: the phase difference
    sum_j dc_j phi_j(f_e) at every edge, formed from a chunk's anchor values,
    scaled derivatives and edge offsets as the device forms it (degree-10
    Taylor form in x = (f_e - f_a) / S), equals the direct basis sum within
    the chunk's remainder bound sum_j |dc_j| bnd_j (plus the FP32 storage of
    the table entries).  dc from coefficient differences of real parameter
    pairs (the library's own coefficient code), near the fiducial and far
    from it; near it, nearly every chunk stays under the device's 1e-6-cycle
    threshold."""
    wl = si.config2() if which == "cfg2" else si.config1()
    out = _run(harness, "hetchunks", repr(wl.f_min), repr(wl.f_max), repr(wl.df), nb, spacing)
    nc, nbasis, npoly, rows = out["nc"], out["nbasis"], out["poly"], out["row"]
    # the tables are FP32: parse the printed values back to the exact floats
    ct = np.array(out["ct"], dtype=np.float32).astype(np.float64).reshape(out["rows"], nc)
    dfe = np.array(out["dfe"], dtype=np.float32).astype(np.float64).reshape(nc, 32)
    fe = np.array(out["fe"])
    assert nc == (out["nb"] + 30) // 31

    def row(name, j=0):
        return ct[rows[name] + j]

    val = np.array([row("val_hi", j) + row("val_lo", j) for j in range(nbasis)])  # [j][q]
    d1 = np.array([row("d1_hi", j) + row("d1_lo", j) for j in range(nbasis)])
    poly = np.array([[row("poly", m * nbasis + j) for j in range(nbasis)] for m in range(npoly)])  # [m][j][q]
    bnd = np.array([row("bnd", j) for j in range(nbasis)])
    inv_s = row("inv_s")
    fa = row("fa_hi") + row("fa_lo")
    th0 = (1.975, 0.8, 0.01, -0.02, 300.0, 500.0)
    pairs = {"near": [(1.975 * (1 + 1e-5), 0.8004, 0.0101, -0.0199, 310.0, 490.0)],
             "far": [(1.6, 0.55, -0.04, 0.04, 4000.0, 100.0)]}
    c0 = np.array(_run(harness, "coeffs", *[repr(v) for v in th0])["c"])
    for kind, ths in pairs.items():
        for th in ths:
            dc = np.array(_run(harness, "coeffs", *[repr(v) for v in th])["c"]) - c0
            R = np.abs(dc) @ bnd  # [q]
            anchored = 0
            for q in range(nc):
                e = np.arange(31 * q, min(31 * q + 31, out["nb"]) + 1)
                assert abs(fe[e[0]] - fa[q]) <= 1e-9 * fe[e[0]]
                direct = dc @ _basis(fe[e])
                x = dfe[q, : e.size] * inv_s[q]
                assert np.all(x >= -1e-6) and np.all(x <= 1 + 1e-6)
                a = [dc @ val[:, q], dc @ d1[:, q]] + [dc @ poly[m, :, q] for m in range(npoly)]
                taylor = a[0] + sum(a[n] * x ** n for n in range(1, npoly + 2))
                storage = 1e-6 * sum(abs(v) for v in a[1:]) + 1e-12 * abs(a[0]) + 1e-12
                assert np.all(np.abs(taylor - direct) <= R[q] + storage), (kind, q, np.abs(taylor - direct).max(), R[q])
                anchored += R[q] <= 1e-6
            if kind == "near" and which == "cfg2":  # 5,000 narrow bins: the Taylor path nearly everywhere
                assert anchored >= 0.9 * nc, (anchored, nc)


def test_nufft_gather_pieces_cover_every_entry_once(harness):
    """The time pass's gather pieces: every grid point's entries, in order,
    cut into runs of at most 31 consecutive edges; the point list names each
    point with entries once, with its pieces contiguous."""
    wl = si.config2()
    edges, _ = L.phase_bound_edges(wl.freqs, 5000)
    stdin = f"{edges.size}\n" + " ".join(repr(float(v)) for v in edges)
    r = subprocess.run([harness, "nufftpieces", "2000", repr(0.2 / 2000)], input=stdin, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    out = json.loads(r.stdout)
    ptr, edge, piece, point, M = out["ptr"], out["edge"], out["piece"], out["point"], out["M"]
    assert len(ptr) == M + 1
    seen = np.zeros(ptr[-1], dtype=int)
    nonempty = [l for l in range(M) if ptr[l + 1] > ptr[l]]
    assert [p[0] for p in point] == nonempty
    for l, p0, npc in point:
        k = ptr[l]
        for p in piece[p0:p0 + npc]:
            k0, n, e0 = p
            assert k0 == k and 1 <= n <= out["max_piece"] and e0 == edge[l] + (k0 - ptr[l])
            seen[k0:k0 + n] += 1
            k += n
        assert k == ptr[l + 1]
    assert np.all(seen == 1)
    assert sum(npc for _, _, npc in point) == len(piece)


def test_nufft_fft_stage_twiddles_reproduce_the_dft(harness):
    """The time pass's radix-2 FFT as the device runs it: bit-reversed input,
    spans 1..16 inside 32-point blocks (each lane pairs with lane ^ h, the
    lower point adding w x partner, the upper subtracting), then the wider
    spans in shared memory, twiddles read from the host's stage-major table
    at h - 1 + p.  Against numpy's inverse-sign DFT of the natural-order
    input, to FP32 accuracy."""
    wl = si.config2()
    edges, _ = L.phase_bound_edges(wl.freqs, 5000)
    stdin = f"{edges.size}\n" + " ".join(repr(float(v)) for v in edges)
    r = subprocess.run([harness, "nufftpieces", "2000", repr(0.2 / 2000)], input=stdin, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    out = json.loads(r.stdout)
    M = out["M"]
    tw = np.array([complex(a, b) for a, b in out["tw"]], dtype=np.complex64)
    assert tw.size == M
    lg = M.bit_length() - 1
    rng = np.random.default_rng(4)
    nat = (rng.standard_normal(M) + 1j * rng.standard_normal(M)).astype(np.complex64)
    rev = np.array([int(format(l, f"0{lg}b")[::-1], 2) for l in range(M)])
    g = np.empty(M, dtype=np.complex64)
    g[rev] = nat
    lane = np.arange(32)
    for blk in range(M // 32):
        x = g[blk * 32:(blk + 1) * 32].copy()
        h = 1
        while h < 32:
            w = tw[h - 1 + (lane & (h - 1))]
            p = x[lane ^ h]
            x = np.where((lane & h) == 0, x + w * p, p - w * x).astype(np.complex64)
            h <<= 1
        g[blk * 32:(blk + 1) * 32] = x
    h = 32
    while h < M:
        b = np.arange(M // 2)
        pos = b & (h - 1)
        i = ((b - pos) << 1) + pos
        j = i + h
        t = tw[h - 1 + pos] * g[j]
        gi = g[i].copy()
        g[j] = gi - t
        g[i] = gi + t
        h <<= 1
    want = np.fft.ifft(nat.astype(np.complex128)) * M
    assert np.abs(g - want).max() <= 2e-6 * np.abs(want).max(), np.abs(g - want).max() / np.abs(want).max()
