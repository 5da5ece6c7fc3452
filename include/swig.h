/*
 * swig.h -- C-ABI of libswig, a GB300-native (sm_103a) Slice-within-Gibbs
 * nested sampler for compact-binary gravitational-wave parameter estimation.
 *
 * The calls follow the paper's statement of the problem: set data, PSDs,
 * detectors and prior; run nested sampling; return posterior samples and the
 * log-evidence.  Citations are to "Ab Initio Real-Time Gravitational-Wave
 * Parameter Estimation" (arXiv 2607.28265) by section / equation / table.
 *
 * Conventions for every call:
 *   - Every function returns SWIG_OK (0) or a negative SWIG_E_* code and never
 *     throws; swig_last_error() gives a message for the last failure on a
 *     context (valid until the next call on that context).
 *   - Host arrays passed in are COPIED; the caller keeps ownership.  Output
 *     buffers are caller-allocated.
 *   - "_dev" variants take device pointers (to memory of the context's device)
 *     and a cudaStream_t passed as void*; they enqueue work and return without
 *     synchronising unless stated.
 *   - A context is not thread-safe; distinct contexts may be used concurrently.
 *   - The 13-vector theta has slots, in order:
 *       0 Mc [Msun] (detector-frame chirp mass), 1 q = m2/m1 <= 1,
 *       2 chi1, 3 chi2 (aligned dimensionless spins), 4 Lambda1, 5 Lambda2,
 *       6 d_L [Mpc], 7 iota [rad], 8 psi [rad], 9 RA [rad], 10 Dec [rad],
 *       11 t_c [s] (relative to the reference time), 12 phi_c [rad].
 */
#ifndef SWIG_H
#define SWIG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SWIG_OK 0
#define SWIG_E_ARG (-1)      /* invalid argument (null pointer, size, range) */
#define SWIG_E_STATE (-2)    /* call out of order (e.g. run before data)     */
#define SWIG_E_NOMEM (-3)    /* host or device allocation failed             */
#define SWIG_E_CUDA (-4)     /* CUDA runtime error                           */
#define SWIG_E_TIMEOUT (-5)  /* a bounded device wait expired                */
#define SWIG_E_NUMERIC (-6)  /* non-finite or non-positive input values      */

/* ---- enumerations ------------------------------------------------------ */
#define SWIG_N_PARAMS 13
#define SWIG_MAX_DET 4

enum swig_prior_kind {       /* Table I prior families, on [lo, hi]          */
  SWIG_PRIOR_UNIFORM = 0,    /* p(x) = const                                 */
  SWIG_PRIOR_SINE = 1,       /* p(x) ~ sin x   (inclination)                 */
  SWIG_PRIOR_COSINE = 2,     /* p(x) ~ cos x   (declination)                 */
  SWIG_PRIOR_POWER2 = 3      /* p(x) ~ x^2     (luminosity distance)         */
};
enum swig_param_mode {
  SWIG_MODE_SAMPLE = 0,      /* sampled by the Gibbs kernel                  */
  SWIG_MODE_FIXED = 1,       /* held at `value`                              */
  SWIG_MODE_MARG = 2         /* marginalised (phi_c, d_L or t_c; see below)  */
};
enum swig_likelihood { SWIG_LIKE_FULL = 0, SWIG_LIKE_HET = 1 };
enum swig_precision { SWIG_PREC_FP64 = 0, SWIG_PREC_MIXED = 1 };
enum swig_proposal { SWIG_PROPOSAL_COV = 0, SWIG_PROPOSAL_LEARNED = 1 };

/* One slot of the 13-vector: prior family and bounds (Table I), mode, and the
 * Gibbs block it belongs to (Sec. 3.2; blocks are swept in increasing id). */
typedef struct swig_param {
  int kind;
  double lo, hi;
  int mode;
  double value;
  int block;
} swig_param;

/* Sampler hyper-parameters (Table II): live points m, deletions k per
 * iteration, Gibbs sweeps M, slice steps per dimension of each block, the
 * termination threshold on log Z_live - log Z_dead (Sec. 3.2: -3). */
typedef struct swig_sampler_cfg {
  int nlive;
  int nrep;
  int sweeps;
  int steps_per_dim;
  uint64_t seed;
  int likelihood;       /* swig_likelihood */
  int precision;        /* swig_precision  */
  int proposal;         /* swig_proposal   */
  int het_bins;         /* heterodyned bins (SWIG_LIKE_HET)              */
  int het_spacing;      /* 0 = equal maximum phase change, 1 = geometric */
  double dlogz;         /* termination threshold, e.g. -3                */
  int max_iter;         /* safety cap on outer iterations                */
  double het_fiducial[SWIG_N_PARAMS]; /* theta of the reference waveform  */
  /* SWIG_PROPOSAL_LEARNED (0 selects the default in brackets):            */
  double learn_mix;     /* probability of a learned direction [0.5]      */
  double learn_lr;      /* Adam learning rate [1e-3]                     */
  int learn_steps;      /* Adam steps per retraining [50; 4x at start]   */
  int learn_interval;   /* NS iterations between retrainings [8]         */
  /* t_c marginalised (slot 11 SWIG_MODE_MARG; heterodyned likelihood only,
   * het_bins <= 16384): nodes of the midpoint grid over the uniform t_c
   * prior [lo, hi], t_j = lo + (j + 1/2)(hi - lo)/tmarg_nodes, 1..65536.
   * The spacing should resolve the t_c posterior (its width is roughly
   * 1 / (2 pi SNR sigma_f), sigma_f the spread of the signal's frequencies).
   * With 64..4096 nodes the time pass is a non-uniform FFT on M >= 2 nodes
   * grid points (a power of two) whose grid, twiddles and edge products share
   * a CTA's shared memory with the sampler's state: about 8 (het_bins + 1) +
   * 16 M bytes plus ~12 KB must fit in 220 KB, else swig_run returns
   * SWIG_E_ARG (e.g. 5000 bins: up to 4096 nodes). */
  int tmarg_nodes;
  /* 1: evaluate every proposal in full, also for the blocks that only move
   * the projection factors (d_L, iota, psi, phi_c), which otherwise reuse the
   * chain's cached per-detector sums of its last full evaluation (exact in C_i,
   * see Sec. 3.2 on fast and slow blocks).  A verification switch: the cached
   * and uncached samplers must agree in distribution.  0 = the cache. */
  int cache_off;
  /* Launch shape of the full-grid mixed-precision sampler (0 selects the
   * default in brackets; swig_autotune picks them per problem): slice parts,
   * the number of sweep units each CTA's share of a proposal is split into,
   * 1..4 [1]; stepout_one_end 1 steps a slice bracket out one end at a time
   * instead of both ends in flight [0].  Both leave the evaluations and
   * results the same up to the grouping of the per-part FP32 sums. */
  int flow_parts;
  int stepout_one_end;
} swig_sampler_cfg;

typedef struct swig_result {
  double logz, logz_err, info, ess, wall_s;
  int64_t n_dead, n_iter, n_evals, n_sweep_evals;
  int status;
} swig_result;

typedef struct swig_ctx swig_ctx;  /* opaque; owned by the library */

/* ---- context ----------------------------------------------------------- */
/* Create a context bound to CUDA device `cuda_device`.  *out is set on success. */
int swig_create(swig_ctx** out, int cuda_device);
/* Free the context and every device buffer it owns.  NULL is a no-op. */
void swig_destroy(swig_ctx* ctx);
/* Message for the last failure on ctx ("" if none).  NULL ctx gives the
 * message of the last failed swig_create in this thread. */
const char* swig_last_error(const swig_ctx* ctx);

/* ---- problem definition (Sec. 3.1) ------------------------------------- */
/* Frequency grid f_k = k df for k = ceil(f_min/df) .. floor(f_max/df), both
 * ends inclusive.  Requires 0 < f_min < f_max, df > 0, at most 2^22 bins. */
int swig_set_grid(swig_ctx* ctx, double f_min, double f_max, double df);
/* Detector `idx` (0 <= idx < SWIG_MAX_DET; detectors must be set
 * contiguously from 0): vertex position [m] and unit arm vectors in the
 * Earth-fixed frame.  The detector tensor is D = (x x^T - y y^T) / 2. */
int swig_set_detector(swig_ctx* ctx, int idx, const double vertex_m[3],
                      const double x_arm[3], const double y_arm[3]);
/* Greenwich mean sidereal time [rad] at the reference time (fixes the Earth's
 * orientation for antenna patterns and delays; Sec. 4.1). */
int swig_set_time_ref(swig_ctx* ctx, double gmst_rad);
/* Frequency-domain strain of detector `det` on the grid: n complex values as
 * 2n doubles (re, im interleaved), time origin at the reference time.
 * n must equal the number of grid bins.  Non-finite values -> SWIG_E_NUMERIC. */
int swig_set_data(swig_ctx* ctx, int det, const double* re_im, int64_t n);
/* One-sided noise PSD S_n(f) [1/Hz] of detector `det` on the grid (n values,
 * all finite and > 0, else SWIG_E_NUMERIC). */
int swig_set_psd(swig_ctx* ctx, int det, const double* psd, int64_t n);
/* Prior: exactly SWIG_N_PARAMS slots (Table I).  Requires lo < hi for sampled
 * slots.  Three slots may be SWIG_MODE_MARG (Sec. 3.1, App. A): phi_c (slot
 * 12, closed-form log I0), d_L (slot 6, uniform or power-law-2 prior on
 * 0 < lo < hi, quadrature; full-grid likelihood only) and t_c (slot 11,
 * uniform prior, grid sum over tmarg_nodes time shifts; heterodyned
 * likelihood only).  The likelihood ignores the theta value of a
 * marginalised slot; the sampler's returned samples carry a post-hoc draw
 * from its conditional for d_L and t_c.  Bad kinds or ranges -> SWIG_E_ARG. */
int swig_set_prior(swig_ctx* ctx, const swig_param* params, int n_params);
/* Sampler configuration (Table II); validated here (nlive > nrep >= 1, ...). */
int swig_set_sampler(swig_ctx* ctx, const swig_sampler_cfg* cfg);

/* ---- likelihood (Eq. 2) ------------------------------------------------- */
/* logL(theta) = -1/2 sum_i <d_i - h_i | d_i - h_i>_i (Eq. 2, without the
 * constant normalisation), or, when phi_c is SWIG_MODE_MARG, the phase-
 * marginalised form log I0(|Z|) - 1/2 sum <h|h> - 1/2 sum <d|d> (Sec. 3.1).
 * theta: n x 13 doubles (row-major, host).  out_logl: n doubles (host).
 * Precision and likelihood type follow the sampler configuration (FULL and
 * MIXED if none was set).  n == 0 is a no-op; n > 2^20 -> SWIG_E_ARG.
 * With SWIG_LIKE_HET the heterodyned (relative-binning) approximation of
 * Sec. 3.4 is evaluated instead: the grid is cut into het_bins bins of equal
 * maximum phase change (het_spacing 0; 1 = geometric), edges snapped to grid
 * frequencies; summary data A0, A1, B0, B1 of the fiducial waveform
 * het_fiducial are formed once in FP64 (phi_c set to 0 when marginalised);
 * h/h0 is taken linear in each bin (value at the centre, slope), so
 *   <d|h> ~ Re sum_b (A0 r0 + A1 r1),  <h|h> ~ sum_b (B0 |r0|^2 + 2 B1 Re(r0 r1*)).
 * The per-bin contraction is FP32 with double-float phase differences; the
 * precision setting does not apply.  An invalid fiducial -> SWIG_E_ARG.
 * With d_L marginalised: the marginal over its prior (64-node quadrature).
 * With t_c marginalised (heterodyned only): the templates are built at the
 * fiducial's t_c, Z is formed at each of the tmarg_nodes grid nodes by
 * rotating the bin-edge ratios, and the result is
 * log((1/N_t) sum_j exp(l_j)) - <h|h>/2 - <d|d>/2 with l_j = log I0(|Z_j|)
 * (or Re Z_j), <h|h> taken once at the fiducial's t_c. */
int swig_loglike_batch(swig_ctx* ctx, const double* theta, int64_t n, double* out_logl);
/* Same with device pointers on the context's device, enqueued on `stream`
 * (cudaStream_t).  Uses the context's scratch buffers, so calls on one
 * context must not overlap. */
int swig_loglike_batch_dev(swig_ctx* ctx, const double* theta_dev, int64_t n,
                           double* out_logl_dev, void* stream);

/* ---- likelihood without allocation ------------------------------------ */
/* The same batched likelihood as swig_loglike_batch_dev (mixed precision),
 * for callers that cannot allocate device memory once they are running: a
 * latency-critical loop with all memory reserved up front, a host runtime that
 * forbids cudaMalloc/cudaFree after start-up, or a process whose device memory
 * belongs to another framework's pool.  (The paper has no counterpart; this is
 * a deployment interface of this library.)
 *   - Allocates nothing.  Its scratch is one fixed 8 MiB array in the library's
 *     device image, held on every device that loads the library until the
 *     process exits.  Batches that do not fit return SWIG_E_ARG with the
 *     capacity in the message (about 250 parameter vectors on the 128 s,
 *     three-detector grid); split larger batches.
 *   - Full-grid likelihood only.  The context must already be prepared, for
 *     SWIG_LIKE_FULL and SWIG_PREC_MIXED, by an
 *     earlier swig_loglike_batch / swig_loglike_batch_dev / swig_run call with
 *     the current data (preparation allocates); otherwise SWIG_E_STATE.
 *   - The first call on a device looks up the array's device address (no
 *     allocation); make that first call before any stream capture.
 *   - Every call shares the one scratch array, which keeps the previous
 *     call's contents; nothing in it needs to start at zero.  Calls that
 *     overlap on the GPU (other streams, other threads, other contexts in the
 *     same process on the same device) race on it: serialise them.
 * theta_dev: n x 13 doubles; out_logl_dev: n doubles; both device pointers on
 * the context's device.  stream: cudaStream_t (NULL = legacy default stream). */
int swig_loglike_batch_noalloc(swig_ctx* ctx, const double* theta_dev, int64_t n, double* out_logl_dev,
                               void* stream);

/* ---- synthetic data (Sec. 4.1 injections) ------------------------------- */
/* Detector strain of one source theta (13 doubles) on the grid, for every
 * detector set, computed on the device in FP64 with the same TaylorF2 model
 * and projection as the likelihood; plus optional noise (n_det x n x 2
 * doubles, detector-major, NULL for none).  If target_snr > 0, d_L is first
 * rescaled so that the network optimal SNR sqrt(sum_i <h_i|h_i>) equals it
 * (PSDs required).  out_re_im: n_det x n complex as 2 doubles each;
 * theta_out (optional): theta with the d_L actually used.  Needs the grid,
 * detectors and time reference; not the data. */
int swig_inject(swig_ctx* ctx, const double* theta, double target_snr, const double* noise_re_im,
                double* out_re_im, double* theta_out);

/* ---- detector-frame sky parameterisation ------------------------------- */
/* Sample the sky as azimuth (slot 9, uniform on [0, 2 pi]) and zenith (slot 10,
 * sine prior on [0, pi]) about the baseline from detector det_b to detector
 * det_a instead of (RA, Dec) (the detector-frame parameterisation the paper
 * adopts for mixing, Sec. 3.2).  The frame's z axis is the baseline, its x axis
 * the Earth's rotation axis made orthogonal to it; a direction maps to (RA, Dec)
 * at the reference sidereal time.  The prior stays isotropic, so evidences and
 * posteriors are those of the equatorial parameterisation; samples are reported
 * as (RA, Dec).  Both slots must be sampled in one Gibbs block (checked when
 * the prior is used: SWIG_E_ARG).  det_a = det_b = -1 restores (RA, Dec). */
int swig_set_sky_frame(swig_ctx* ctx, int det_a, int det_b);

/* ---- prior transform (Table I) ---------------------------------------- */
/* Map n unit-cube points (n x n_sampled doubles, sampled slots in slot order)
 * to full 13-vectors theta (n x 13). */
int swig_prior_transform(swig_ctx* ctx, const double* u, int64_t n, double* theta);

/* ---- nested sampling (Sec. 2.2, 2.3, 3.2) ------------------------------ */
/* Run nested sampling to termination (Sec. 3.2: log Z_live - log Z_dead <
 * dlogz) or to about max_iter iterations, on the device.  Requires the prior
 * and the sampler configuration; nlive <= 8192, nrep <= 2048 and at most 32
 * chains per CTA of the persistent kernel.  SWIG_E_TIMEOUT if a bounded
 * device wait expired (the context stays usable). */
int swig_run(swig_ctx* ctx, swig_result* out);
/* Launch-shape tuning for this context's problem (grid, detectors, prior,
 * sampler settings): runs `iters` NS iterations from the configured seed
 * with each candidate shape (flow_parts, stepout_one_end) in (1, 0), (1, 1),
 * (2, 0), (3, 0), measures full-grid evaluations per second of the
 * persistent kernel (CUDA events), and keeps the fastest in the context's
 * sampler settings for later runs.  out (optional): out[0] the number of
 * candidates, then per candidate flow_parts, stepout_one_end and the rate
 * (min(n, 1 + 3 x candidates) values).  Only the full-grid mixed-precision
 * covariance-proposal sampler has a launch shape: for other settings it
 * writes out[0] = 0 and changes nothing.  Errors as swig_run; the settings
 * are restored on an error. */
int swig_autotune(swig_ctx* ctx, int iters, double* out, int n);
/* Run nested sampling for a campaign of n_ctx events (config 4), each a
 * context set up as for swig_run; outs[i] receives event i's result and each
 * context keeps its samples.  Events that can share a launch (full grid, mixed
 * precision, covariance proposal, same detector count, chains and device) and
 * whose grids are within 1.5x of each other (the events of a launch advance
 * their iterations in step) run up to 4 at a time in one persistent launch: their slices of the
 * grid share each CTA's shared memory and their chains share the control and
 * sweep warps, which keeps the GPU busy while one event's chains wait.  Per
 * event the arithmetic and its order are those of swig_run, so the results
 * are the same; an event's persistent-kernel time in the profile is the
 * shared launch time.  Other events run one after another.  A context may
 * appear once.  Stops at the first failure (that context's error). */
int swig_run_batch(swig_ctx** ctxs, int n_ctx, swig_result* outs);
/* Cap, in polling iterations of ~100 ns, on every spin-wait of the persistent
 * kernel (grid barriers).  Default 1e7.  A wait that reaches the cap makes
 * swig_run return SWIG_E_TIMEOUT instead of hanging. */
int swig_set_wait_limit(swig_ctx* ctx, long long spins);
/* Counters of the last swig_run.  Phase timers measured on the device by the
 * first CTA of the persistent kernel: out[0] rounds, out[1] iteration-
 * boundary seconds, out[2] chain-control seconds, out[3] wait after control,
 * out[4] sweep seconds, out[5] wait after sweep; out[6] total milliseconds of
 * the persistent-kernel launches (CUDA events on the context's stream),
 * out[7] their count; over the context's lifetime: out[8] kernel launches,
 * out[9] bytes copied host->device, out[10] device->host; out[11] bin-detector
 * evaluations of the last run (full-grid evaluations x detectors x bins);
 * out[12..16] clock cycles the first chain's control spent on pending results,
 * new slice steps, proposals, projection-only evaluations and full-evaluation
 * set-up, out[17..19] the counts of the last three; out[20] milliseconds of
 * learned-proposal training (targets, Adam steps, output rows; CUDA events)
 * and out[21] the number of retrainings; out[22..24] for the first CTA's
 * sweep warps: (chain, slice) units evaluated, clock cycles spent in them and
 * cycles spent polling for work.  Then, for each CTA s of the last run's
 * persistent kernel (single-event sampler), out[25 + 4 s .. 25 + 4 s + 3]:
 * its sweep warps' units, their cycles in units and polling, and its control
 * warp's cycles advancing chains.  In the heterodyned sampler a unit is one
 * contraction of a chain's proposal by the whole CTA (bin pass, time pass,
 * reductions), and the polling cycles are those the contracting warps wait
 * for the control warp (control and epilogue).  Writes min(n, 25 + 4 x CTAs)
 * values. */
int swig_get_profile(swig_ctx* ctx, double* out, int n);
/* Use `stream` (a cudaStream_t on the context's device, owned by the caller)
 * for all later work of this context; NULL restores a private stream. */
int swig_set_stream(swig_ctx* ctx, void* stream);
/* Dead points of the last run (theta n x 13, logL, log-weight normalised so
 * that logsumexp(logw) = log Z).  With cap == 0 only *n_out is set. */
int swig_get_samples(swig_ctx* ctx, double* theta, double* logl, double* logw,
                     int64_t cap, int64_t* n_out);

/* ---- learned slice proposal (SWIG_PROPOSAL_LEARNED) --------------------- */
/* The paper draws slice directions from the live covariance (Sec. 2.3, Eq. 3)
 * and learns nothing; this network is the library's optional alternative and
 * these calls expose its pieces for verification.  Model: 13 -> 256 -> 256 ->
 * 26 with SiLU; input a live point standardised by the live set's mean and
 * standard deviation (zero beyond the d sampled dimensions); output a
 * direction u (13) and log-widths s (13).  Training targets per live point:
 * the leading eigenvector e1 of the correlation matrix of its 2d nearest live
 * neighbours (standardised Euclidean distance, ties by index) and their log
 * standard deviations t; loss = mean(1 - (u_hat . e1)^2 + |s - t|^2) over the
 * sampled dimensions.  Matrix products take bfloat16 operands (round to
 * nearest even) and accumulate in FP32; master weights and Adam are FP32.
 * A sampler run retrains every learn_interval iterations on the current live
 * set and draws, with probability learn_mix, the direction
 * exp(s_b) * u_b / |u_b| of the Gibbs block from the output row of a live
 * point picked uniformly from that snapshot.
 * Parameter vector (SWIG_MLP_PARAMS floats, host): W1 [13][256], b1 [256],
 * W2 [256][256], b2 [256], W3 [256][26], b3 [26], row = input unit.
 * All buffers below are host arrays; n <= 8192, 1 <= d <= 13. */
#define SWIG_MLP_PARAMS 76058
/* Initial parameters: W ~ N(0, 1/fan_in) by Philox-4x32-10 (counter
 * (column, row, layer, 9), key = seed) and Box-Muller; biases 0. */
int swig_mlp_init(swig_ctx* ctx, uint64_t seed, float* params_out);
/* Outputs (n x 26) of n standardised inputs x_std (n x 13). */
int swig_mlp_forward(swig_ctx* ctx, const float* params, const float* x_std, int64_t n, float* out);
/* Loss and its gradient (SWIG_MLP_PARAMS floats) for inputs x_std (n x 13)
 * and targets tdir, tls (n x 13, zero beyond d). */
int swig_mlp_loss_grad(swig_ctx* ctx, const float* params, const float* x_std, const float* tdir,
                       const float* tls, int64_t n, int d, double* loss_out, float* grad_out);
/* Training targets of n live points (live_u: n x d doubles in the unit cube):
 * tdir, tls (n x 13 floats); nbr (optional, n x 26 ints): the 2d neighbour
 * indices in distance order.  Requires 2d < n. */
int swig_mlp_targets(swig_ctx* ctx, const double* live_u, int64_t n, int d, float* tdir, float* tls, int* nbr);
/* `steps` Adam steps (fresh Adam state, learning rate lr) from params_inout on
 * the targets of live_u; params_inout receives the trained parameters and
 * out_rows (optional, n x 26) the trained network's outputs on live_u. */
int swig_mlp_train(swig_ctx* ctx, const double* live_u, int64_t n, int d, int steps, double lr,
                   float* params_inout, float* out_rows);

#ifdef __cplusplus
}
#endif
#endif /* SWIG_H */
