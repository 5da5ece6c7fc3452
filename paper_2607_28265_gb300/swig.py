"""ctypes binding of libswig (the C-ABI in include/swig.h).

Argument marshalling only: every step of the likelihood and the sampler runs in
the library's CUDA kernels.  Loading fails loudly when the library has not
been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libswig.so")

SWIG_OK, SWIG_E_ARG, SWIG_E_STATE, SWIG_E_NOMEM, SWIG_E_CUDA, SWIG_E_TIMEOUT, SWIG_E_NUMERIC = 0, -1, -2, -3, -4, -5, -6
N_PARAMS = 13
MAX_DET = 4
LIKE_FULL, LIKE_HET = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
PROPOSAL_COV, PROPOSAL_LEARNED = 0, 1

# Every entry point declared in include/swig.h, with ctypes signatures.
_c_int, _c_double, _c_i64, _c_u64, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
MLP_PARAMS = 76058


class SwigParam(ctypes.Structure):
    _fields_ = [("kind", _c_int), ("lo", _c_double), ("hi", _c_double), ("mode", _c_int),
                ("value", _c_double), ("block", _c_int)]


class SwigSamplerCfg(ctypes.Structure):
    _fields_ = [("nlive", _c_int), ("nrep", _c_int), ("sweeps", _c_int), ("steps_per_dim", _c_int),
                ("seed", _c_u64), ("likelihood", _c_int), ("precision", _c_int), ("proposal", _c_int),
                ("het_bins", _c_int), ("het_spacing", _c_int), ("dlogz", _c_double), ("max_iter", _c_int),
                ("het_fiducial", _c_double * N_PARAMS), ("learn_mix", _c_double), ("learn_lr", _c_double),
                ("learn_steps", _c_int), ("learn_interval", _c_int), ("tmarg_nodes", _c_int),
                ("cache_off", _c_int), ("flow_parts", _c_int), ("stepout_one_end", _c_int)]


class SwigResult(ctypes.Structure):
    _fields_ = [("logz", _c_double), ("logz_err", _c_double), ("info", _c_double), ("ess", _c_double),
                ("wall_s", _c_double), ("n_dead", _c_i64), ("n_iter", _c_i64), ("n_evals", _c_i64),
                ("n_sweep_evals", _c_i64), ("status", _c_int)]


SIGNATURES = {
    "swig_create": (_c_int, [ctypes.POINTER(_vp), _c_int]),
    "swig_destroy": (None, [_vp]),
    "swig_last_error": (ctypes.c_char_p, [_vp]),
    "swig_set_grid": (_c_int, [_vp, _c_double, _c_double, _c_double]),
    "swig_set_detector": (_c_int, [_vp, _c_int, _dp, _dp, _dp]),
    "swig_set_time_ref": (_c_int, [_vp, _c_double]),
    "swig_set_data": (_c_int, [_vp, _c_int, _dp, _c_i64]),
    "swig_set_psd": (_c_int, [_vp, _c_int, _dp, _c_i64]),
    "swig_set_prior": (_c_int, [_vp, ctypes.POINTER(SwigParam), _c_int]),
    "swig_set_sampler": (_c_int, [_vp, ctypes.POINTER(SwigSamplerCfg)]),
    "swig_loglike_batch": (_c_int, [_vp, _dp, _c_i64, _dp]),
    "swig_loglike_batch_dev": (_c_int, [_vp, _vp, _c_i64, _vp, _vp]),
    "swig_prior_transform": (_c_int, [_vp, _dp, _c_i64, _dp]),
    "swig_run": (_c_int, [_vp, ctypes.POINTER(SwigResult)]),
    "swig_autotune": (_c_int, [_vp, _c_int, _dp, _c_int]),
    "swig_set_wait_limit": (_c_int, [_vp, ctypes.c_longlong]),
    "swig_get_profile": (_c_int, [_vp, _dp, _c_int]),
    "swig_set_stream": (_c_int, [_vp, _vp]),
    "swig_inject": (_c_int, [_vp, _dp, _c_double, _dp, _dp, _dp]),
    "swig_loglike_batch_noalloc": (_c_int, [_vp, _vp, _c_i64, _vp, _vp]),
    "swig_get_samples": (_c_int, [_vp, _dp, _dp, _dp, _c_i64, ctypes.POINTER(_c_i64)]),
    "swig_set_sky_frame": (_c_int, [_vp, _c_int, _c_int]),
    "swig_run_batch": (_c_int, [ctypes.POINTER(_vp), _c_int, ctypes.POINTER(SwigResult)]),
    "swig_mlp_init": (_c_int, [_vp, _c_u64, _fp]),
    "swig_mlp_forward": (_c_int, [_vp, _fp, _fp, _c_i64, _fp]),
    "swig_mlp_loss_grad": (_c_int, [_vp, _fp, _fp, _fp, _fp, _c_i64, _c_int, _dp, _fp]),
    "swig_mlp_targets": (_c_int, [_vp, _dp, _c_i64, _c_int, _fp, _fp, _ip]),
    "swig_mlp_train": (_c_int, [_vp, _dp, _c_i64, _c_int, _c_int, _c_double, _fp, _fp]),
}

_lib = None


class SwigError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libswig error {code}: {msg}")
        self.code = code


def load_library(path: str = LIB_PATH):
    """Load libswig.so (built by __graft_entry__.build()); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libswig.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fptr(a):
    return a.ctypes.data_as(_fp)


@dataclass
class RunResult:
    logz: float
    logz_err: float
    info: float
    ess: float
    wall_s: float
    n_dead: int
    n_iter: int
    n_evals: int
    n_sweep_evals: int
    status: int


class Context:
    """One libswig context on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        h = _vp()
        rc = self.lib.swig_create(ctypes.byref(h), int(device))
        if rc != SWIG_OK:
            raise SwigError(rc, self.lib.swig_last_error(None).decode())
        self.h = h
        self.n_bins = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.swig_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != SWIG_OK:
            raise SwigError(rc, self.lib.swig_last_error(self.h).decode())

    def call(self, name, *args):
        """Raw call returning the status code (for tests of error paths)."""
        return getattr(self.lib, name)(self.h, *args)

    # ---- problem definition ------------------------------------------------
    def set_grid(self, f_min, f_max, df):
        self._check(self.lib.swig_set_grid(self.h, f_min, f_max, df))
        import math
        self.n_bins = int(math.floor(f_max / df + 1e-9)) - int(math.ceil(f_min / df - 1e-9)) + 1

    def set_detector(self, idx, vertex, x_arm, y_arm):
        v, x, y = (np.ascontiguousarray(a, dtype=np.float64) for a in (vertex, x_arm, y_arm))
        self._check(self.lib.swig_set_detector(self.h, idx, _ptr(v), _ptr(x), _ptr(y)))

    def set_time_ref(self, gmst):
        self._check(self.lib.swig_set_time_ref(self.h, float(gmst)))

    def set_data(self, det, data):
        d = np.ascontiguousarray(np.asarray(data, dtype=np.complex128)).view(np.float64)
        self._check(self.lib.swig_set_data(self.h, det, _ptr(d), d.size // 2))

    def set_psd(self, det, psd):
        s = np.ascontiguousarray(psd, dtype=np.float64)
        self._check(self.lib.swig_set_psd(self.h, det, _ptr(s), s.size))

    def set_prior(self, params):
        arr = (SwigParam * N_PARAMS)()
        for i, p in enumerate(params):
            arr[i] = SwigParam(p.kind, p.lo, p.hi, p.mode, p.value, p.block)
        self._check(self.lib.swig_set_prior(self.h, arr, len(params)))

    def set_sampler(self, nlive, nrep, sweeps=1, steps_per_dim=5, seed=0, likelihood=LIKE_FULL,
                    precision=PREC_MIXED, proposal=PROPOSAL_COV, het_bins=0, het_spacing=0, dlogz=-3.0,
                    max_iter=100000, het_fiducial=None, learn_mix=0.0, learn_lr=0.0, learn_steps=0,
                    learn_interval=0, tmarg_nodes=0, cache_off=0, flow_parts=0, stepout_one_end=0):
        """swig_set_sampler: the fields of swig_sampler_cfg (include/swig.h).

        nlive / nrep: live points m and deletions k per iteration; sweeps (M)
        and steps_per_dim: Gibbs sweeps per replacement and slice steps per
        dimension of a block; likelihood LIKE_FULL or LIKE_HET with het_bins,
        het_spacing (0 equal phase change, 1 geometric) and het_fiducial (13
        values); precision PREC_FP64 or PREC_MIXED; proposal PROPOSAL_COV or
        PROPOSAL_LEARNED with learn_* (0 = library default); tmarg_nodes: grid
        nodes over the t_c prior when t_c is marginalised (heterodyned only);
        cache_off=1 evaluates projection-only proposals in full (no reuse of
        the chain's cached per-detector sums).
        """
        cfg = SwigSamplerCfg()
        cfg.nlive, cfg.nrep, cfg.sweeps, cfg.steps_per_dim = nlive, nrep, sweeps, steps_per_dim
        cfg.seed, cfg.likelihood, cfg.precision, cfg.proposal = seed, likelihood, precision, proposal
        cfg.het_bins, cfg.het_spacing, cfg.dlogz, cfg.max_iter = het_bins, het_spacing, dlogz, max_iter
        if het_fiducial is not None:
            for i, v in enumerate(het_fiducial):
                cfg.het_fiducial[i] = float(v)
        cfg.learn_mix, cfg.learn_lr = float(learn_mix), float(learn_lr)
        cfg.learn_steps, cfg.learn_interval = int(learn_steps), int(learn_interval)
        cfg.tmarg_nodes = int(tmarg_nodes)
        cfg.cache_off = int(cache_off)
        cfg.flow_parts = int(flow_parts)
        cfg.stepout_one_end = int(stepout_one_end)
        self._check(self.lib.swig_set_sampler(self.h, ctypes.byref(cfg)))

    # ---- likelihood --------------------------------------------------------
    def loglike_batch(self, theta):
        th = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
        out = np.empty(th.shape[0])
        self._check(self.lib.swig_loglike_batch(self.h, _ptr(th), th.shape[0], _ptr(out)))
        return out

    def loglike_batch_dev(self, theta_dev_ptr, n, out_dev_ptr, stream_ptr=0):
        """Device pointers (e.g. torch tensor.data_ptr()) and a raw cudaStream_t."""
        self._check(self.lib.swig_loglike_batch_dev(self.h, _vp(theta_dev_ptr), int(n), _vp(out_dev_ptr),
                                                     _vp(stream_ptr)))

    def inject(self, theta, n_det, target_snr=0.0, noise=None):
        """Detector strains (n_det x n_bins complex) of theta plus optional noise;
        returns (data, theta_used)."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        out = np.empty((n_det, self.n_bins), dtype=np.complex128)
        nz = None
        if noise is not None:
            nz = np.ascontiguousarray(np.asarray(noise, dtype=np.complex128)).view(np.float64)
        th_out = np.empty(N_PARAMS)
        self._check(self.lib.swig_inject(self.h, _ptr(th), float(target_snr), None if nz is None else _ptr(nz),
                                         _ptr(out.view(np.float64)), _ptr(th_out)))
        return out, th_out

    def loglike_batch_noalloc(self, theta_dev_ptr, n, out_dev_ptr, stream_ptr=0):
        """Batched likelihood with the library's fixed scratch (no device
        allocation); the context must have been prepared by an earlier
        likelihood call."""
        self._check(self.lib.swig_loglike_batch_noalloc(self.h, _vp(theta_dev_ptr), int(n), _vp(out_dev_ptr),
                                                         _vp(stream_ptr)))

    def prior_transform(self, u):
        uu = np.ascontiguousarray(np.atleast_2d(u), dtype=np.float64)
        th = np.empty((uu.shape[0], N_PARAMS))
        self._check(self.lib.swig_prior_transform(self.h, _ptr(uu), uu.shape[0], _ptr(th)))
        return th

    # ---- nested sampling ---------------------------------------------------
    def run(self) -> RunResult:
        r = SwigResult()
        self._check(self.lib.swig_run(self.h, ctypes.byref(r)))
        return RunResult(r.logz, r.logz_err, r.info, r.ess, r.wall_s, r.n_dead, r.n_iter, r.n_evals,
                         r.n_sweep_evals, r.status)

    def autotune(self, iters=8):
        """swig_autotune: try the launch shapes for `iters` NS iterations each and
        keep the fastest.  Returns (candidates, chosen): candidates a list of
        (flow_parts, stepout_one_end, full-grid evals/s), chosen the kept
        (flow_parts, stepout_one_end) or None when the settings have no
        launch shape."""
        buf = np.zeros(1 + 3 * 8)
        self._check(self.lib.swig_autotune(self.h, int(iters), buf.ctypes.data_as(_dp), buf.size))
        n = int(buf[0])
        cands = [(int(buf[1 + 3 * i]), int(buf[2 + 3 * i]), float(buf[3 + 3 * i])) for i in range(n)]
        if not cands:
            return cands, None
        best = max(cands, key=lambda t: t[2])
        return cands, (best[0], best[1])

    PROFILE_KEYS = ("rounds", "boundary_s", "control_s", "wait_control_s", "sweep_s", "wait_sweep_s",
                    "persistent_ms", "persistent_launches", "kernel_launches", "h2d_bytes", "d2h_bytes",
                    "bin_det_evals", "cyc_result", "cyc_step", "cyc_prop", "cyc_free", "cyc_setup", "n_free",
                    "n_setup", "n_step", "learn_ms", "learn_rounds", "f_units",
                    "f_unit_cyc", "f_idle_cyc")

    def profile(self):
        out = np.zeros(len(self.PROFILE_KEYS))
        self._check(self.lib.swig_get_profile(self.h, _ptr(out), out.size))
        return dict(zip(self.PROFILE_KEYS, out.tolist()))

    def cta_profile(self, n_ctas):
        """Per-CTA counters of the last run's persistent kernel (n_ctas x 4):
        sweep units, cycles in units, cycles polling, control cycles."""
        out = np.zeros(len(self.PROFILE_KEYS) + 4 * int(n_ctas))
        self._check(self.lib.swig_get_profile(self.h, _ptr(out), out.size))
        return out[len(self.PROFILE_KEYS):].reshape(-1, 4)

    def set_sky_frame(self, det_a=-1, det_b=-1):
        """Sample the sky as (azimuth, zenith) about the det_b -> det_a baseline."""
        self._check(self.lib.swig_set_sky_frame(self.h, int(det_a), int(det_b)))

    def set_stream(self, stream_ptr):
        self._check(self.lib.swig_set_stream(self.h, _vp(stream_ptr)))

    def set_wait_limit(self, spins):
        self._check(self.lib.swig_set_wait_limit(self.h, int(spins)))

    def get_samples(self):
        n = _c_i64(0)
        self._check(self.lib.swig_get_samples(self.h, None, None, None, 0, ctypes.byref(n)))
        th = np.empty((n.value, N_PARAMS))
        ll = np.empty(n.value)
        lw = np.empty(n.value)
        self._check(self.lib.swig_get_samples(self.h, _ptr(th), _ptr(ll), _ptr(lw), n.value, ctypes.byref(n)))
        return th, ll, lw

    # ---- learned slice proposal -------------------------------------------
    def mlp_init(self, seed):
        p = np.empty(MLP_PARAMS, dtype=np.float32)
        self._check(self.lib.swig_mlp_init(self.h, int(seed), _fptr(p)))
        return p

    def mlp_forward(self, params, x_std):
        p, x = _f32(params), _f32(np.atleast_2d(x_std))
        out = np.empty((x.shape[0], 26), dtype=np.float32)
        self._check(self.lib.swig_mlp_forward(self.h, _fptr(p), _fptr(x), x.shape[0], _fptr(out)))
        return out

    def mlp_loss_grad(self, params, x_std, tdir, tls, d):
        p, x, t, l = _f32(params), _f32(x_std), _f32(tdir), _f32(tls)
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        self._check(self.lib.swig_mlp_loss_grad(self.h, _fptr(p), _fptr(x), _fptr(t), _fptr(l), x.shape[0], int(d),
                                                ctypes.byref(loss), _fptr(g)))
        return loss.value, g

    def mlp_targets(self, live_u):
        u = np.ascontiguousarray(live_u, dtype=np.float64)
        n, d = u.shape
        tdir = np.empty((n, 13), dtype=np.float32)
        tls = np.empty((n, 13), dtype=np.float32)
        nbr = np.empty((n, 26), dtype=np.int32)
        self._check(self.lib.swig_mlp_targets(self.h, _ptr(u), n, d, _fptr(tdir), _fptr(tls),
                                              nbr.ctypes.data_as(_ip)))
        return tdir, tls, nbr[:, :2 * d]

    def mlp_train(self, live_u, params, steps, lr=1e-3):
        u = np.ascontiguousarray(live_u, dtype=np.float64)
        n, d = u.shape
        p = _f32(params).copy()
        out = np.empty((n, 26), dtype=np.float32)
        self._check(self.lib.swig_mlp_train(self.h, _ptr(u), n, d, int(steps), float(lr), _fptr(p), _fptr(out)))
        return p, out


def run_batch(contexts):
    """Run a campaign of contexts (swig_run_batch); returns their RunResults."""
    n = len(contexts)
    arr = (_vp * n)(*[c.h for c in contexts])
    res = (SwigResult * n)()
    rc = load_library().swig_run_batch(arr, n, res)
    if rc != SWIG_OK:
        for c in contexts:
            msg = c.lib.swig_last_error(c.h).decode()
            if msg:
                raise SwigError(rc, msg)
        raise SwigError(rc, "swig_run_batch failed")
    return [RunResult(r.logz, r.logz_err, r.info, r.ess, r.wall_s, r.n_dead, r.n_iter, r.n_evals, r.n_sweep_evals,
                      r.status) for r in res]


def context_for_workload(wl, data, psds, gmst, device=0, precision=PREC_MIXED, detectors=None):
    """Convenience: a Context loaded with a workload's grid, detectors, data and prior."""
    import swig_inputs as si

    ctx = Context(device)
    ctx.set_grid(wl.f_min, wl.f_max, wl.df)
    for i, name in enumerate(wl.detectors if detectors is None else detectors):
        ctx.set_detector(i, *si.site_vectors(name))
        ctx.set_data(i, data[i])
        ctx.set_psd(i, psds[i])
    ctx.set_time_ref(gmst)
    ctx.set_prior(wl.params)
    return ctx
