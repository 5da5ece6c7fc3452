// Launch interface between the C-ABI host code and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include "swig_internal.h"

namespace swig {

struct PriorSlot {
  int kind;
  int mode;
  double lo, hi, value;
  double c1, c2;  // SINE: cos lo, cos hi; COSINE: sin lo, sin hi; POWER2: lo^3, hi^3
};

inline PriorSlot make_prior_slot(int kind, int mode, double lo, double hi, double value);

// Detector-frame sky parameterisation: slots 9 and 10 hold the azimuth and
// zenith of the source about the baseline between two detectors (ez, from
// detector b to detector a; ex towards the Earth's north pole), mapped to
// (RA, Dec) at the reference sidereal time before any use.
struct SkyFrame {
  int on;
  double ex[3], ey[3], ez[3];
  double gmst;
};

// Time-marginalised heterodyned likelihood: threads per CTA (one theta or
// one chain per CTA), the largest bin count (the edge products y_e live in
// shared memory) and the shared-memory bytes of those products.
constexpr int kHetTmThreads = 512;
constexpr int kMaxTmBins = 16384;
// Non-uniform FFT time pass: node counts it serves (the direct sum below and
// above), the kernel width in grid points; its grid of M complex values
// follows the edge products in shared memory.
constexpr int kNufftMinNodes = 64;
constexpr int kNufftMaxNodes = 4096;
constexpr int kNufftWidth = 8;
// entries per gather piece (one lane sums a piece)
// (odd, so that the pieces of one grid point start in different banks)
constexpr int kNufftPiece = 31;
// (edge products, then the non-uniform FFT's grid of M and stage-major
// twiddle table of M complex values, then the gather's per-piece partial sums)
inline size_t het_tm_smem_bytes(int n_bins, int nufft_m = 0, int pieces = 0) {
  return (((size_t)n_bins + 1) * 2 * sizeof(float) + 15) / 16 * 16 + (size_t)nufft_m * 4 * sizeof(float) +
         (size_t)pieces * 2 * sizeof(float);
}

// Heterodyned contraction by chunk anchors.  A warp step covers one chunk of
// 32 edges (31 bins).  Per chunk the host tabulates, at its first edge f_a,
// the basis values and first derivative (double-float) and the scaled
// derivatives of orders 2..kHetTaylorDeg (float), as rows of a [HC_ROWS][chunks]
// table; per evaluation the phase difference from the fiducial is anchored
// there in double-float and carried across the chunk by an FP32 Taylor form
// in x = (f_e - f_a) / S (S the chunk's span).  Rows HC_BND + j hold the
// remainder bound of basis j, max |phi_j^(11)| S^11 / 11! over the chunk: an
// evaluation whose sum_j |c_j - c0_j| HC_BND_j exceeds kHetTaylorEps cycles
// takes the chunk edge by edge in double-float instead.
constexpr int kHetChunkEdges = 32;
constexpr float kHetTaylorEps = 1e-6f;
// degree of the chunk Taylor form (wider than the full grid's tiles: a chunk
// of 31 heterodyned bins spans up to ~10 % of its frequency mid-band)
constexpr int kHetTaylorDeg = 10;
constexpr int kHetPoly = kHetTaylorDeg - 1;  // orders 2..kHetTaylorDeg
enum HetChunkRow {
  HC_VAL_HI = 0,
  HC_VAL_LO = NBASIS,
  HC_D1_HI = 2 * NBASIS,
  HC_D1_LO = 3 * NBASIS,
  HC_POLY = 4 * NBASIS,  // HC_POLY + (n - 2) * NBASIS + j: phi_j^(n)(f_a) S^n / n!
  HC_FA_HI = 4 * NBASIS + kHetPoly * NBASIS,
  HC_FA_LO,
  HC_INV_S,
  HC_BND,
  HC_ROWS = HC_BND + NBASIS
};
// Per-evaluation chunk anchor in shared memory: a_1 .. a_kHetTaylorDeg, then
// frac(dP(f_a) + f_a dtau_i) per detector, 1 / S and the exact flag of this
// evaluation.
constexpr int kHetAncStride = 16;
constexpr int kHetAncPhase = kHetPoly + 1;
constexpr int kHetAncInvS = kHetAncPhase + SWIG_MAX_DET;
constexpr int kHetAncExact = kHetAncInvS + 1;
static_assert(kHetAncExact < kHetAncStride, "chunk anchor layout");
// Per-warp shared-memory stage of one chunk's table data (summary data, bin
// widths, edge offsets), filled by cp.async one chunk ahead: bytes per stage.
inline size_t het_stage_bytes(int n_det) { return (size_t)n_det * 32 * (16 + 8) + 2 * 32 * 4; }

// Device buffers owned by a context (all allocated with cudaMalloc).
struct DeviceBuffers {
  // problem data
  float2* data32 = nullptr;      // [n_det][n_bins] scaled D_i (MIXED)
  double2* data64 = nullptr;     // [n_det][n_bins] D_i (FP64)
  double* ftab = nullptr;        // [n_bins][3] f^-1/3, f^1/3, ln f (FP64)
  TileInfo* tiles = nullptr;     // [n_tiles]
  TileBasis* basis = nullptr;    // [n_tiles]
  int* slice_begin = nullptr;    // [n_slices + 1] first bin of each slice
  int* bin_tile = nullptr;       // [n_bins] tile of each bin
  PriorSlot* prior = nullptr;    // [13]
  int* piece_begin = nullptr;    // first bin of each sweep piece, slices concatenated (+ end per slice)
  int* slice_piece = nullptr;    // [n_slices + 1] offset of each slice's entries in piece_begin
  int n_pieces = 0;              // total pieces (work units per theta)
  int max_pieces = 1;            // pieces of the largest slice
  int max_slice_bins = 0;
  // heterodyned likelihood tables (SWIG_LIKE_HET)
  int het_nb = 0;
  float* het_edge_basis = nullptr;  // [2 * NBASIS][N_b + 1] (row per basis function, hi / lo)
  float* het_edge_f = nullptr;      // [2][N_b + 1] (hi row, lo row)
  float* het_inv_width = nullptr;   // [N_b]
  float4* het_coef = nullptr;       // [n_det][N_b]
  float2* het_coefB = nullptr;      // [n_det][N_b]
  int het_nc = 0;                   // chunks of kHetChunkEdges edges
  float* het_chunk = nullptr;       // [HC_ROWS][het_nc] chunk anchor tables
  float* het_dfe = nullptr;         // [het_nc][32] f_e - f_a of each chunk's edges
  EvalRecord* het_fid = nullptr;    // fiducial record
  // time marginalisation on the heterodyned bins (t_c marginalised)
  float2* het_tm_g = nullptr;       // [n_det][N_b + 1] edge weights: Z_i = sum_e g_ie r_i(e)
  float2* het_tm_w = nullptr;       // [N_b + 1] exp(-2 pi i f_e dt), the step between grid nodes
  // ... by non-uniform FFT (L.tm_M > 0): kernel weight of every (grid point,
  // edge) entry in grid-point order, deconvolution 1 / Phi per node, twiddles
  float* het_nu_wt = nullptr;       // [entries]
  float* het_nu_corr = nullptr;     // [N_t]
  float2* het_nu_tw = nullptr;      // [M] stage-major twiddles: span h at h - 1 + p, exp(2 pi i p / (2 h))
  int4* het_nu_piece = nullptr;     // [pieces] (first entry, entries, first edge, 0)
  int4* het_nu_point = nullptr;     // [points] (grid point, first piece, pieces, 0)
  // scratch for batched evaluation, sized for `cap` thetas
  int cap = 0;
  EvalRecord* rec = nullptr;     // [cap]
  float* anchors = nullptr;      // [cap][n_tiles][kAnchorStride]
  float* partials32 = nullptr;   // [cap][n_slices][kPartialStride]
  double* partials64 = nullptr;  // [cap][n_slices][kPartialStride]
  double* theta = nullptr;       // [cap][13] staging for host calls
  double* out = nullptr;         // [cap]
  double* u = nullptr;           // [cap][13]
};

// logL of n thetas (device pointers) into out; kappa_out (optional, n x 8
// doubles) receives the unscaled per-detector sums (re, im) for each theta.
cudaError_t launch_loglike_mixed(const LikeConst& L, const DeviceBuffers& B, const double* theta, int n,
                                 double* out, cudaStream_t st, double* kappa_out = nullptr);
cudaError_t launch_loglike_fp64(const LikeConst& L, const DeviceBuffers& B, const double* theta, int n,
                                double* out, cudaStream_t st, double* kappa_out = nullptr);
// Setup record and detector strain of one theta (FP64) into out [n_det][n_bins].
cudaError_t launch_waveform(const LikeConst& L, const double* theta_dev, EvalRecord* rec_dev, double2* out,
                            cudaStream_t st);
// Post-hoc d_L of n samples of a distance-marginalised run (records in B.rec
// and their kappa sums from the preceding likelihood launch); writes theta[6].
cudaError_t launch_distance_draw(const LikeConst& L, const DeviceBuffers& B, const double* kappa, int n,
                                 long long first, unsigned k0, unsigned k1, double* theta, cudaStream_t st);
// Heterodyned logL of n thetas (device pointers), one warp per theta.
// kappa_out (n x 8) / vv_out (n x 4), optional: the per-detector cache of
// projection-only evaluations (het.cuh het_cache).
// With t_c marginalised (L.tm_n > 0) one CTA of kHetTmThreads per theta
// instead, and ell (optional, n x tm_n) receives each node's log weight.
cudaError_t launch_loglike_het(const LikeConst& L, const DeviceBuffers& B, const double* theta, int n, double* out,
                               cudaStream_t st, double* kappa_out = nullptr, double* vv_out = nullptr,
                               float* ell = nullptr);
// Post-hoc t_c of n time-marginalised samples from their node log weights
// (records of the same samples in B.rec); sample i uses the Philox counter of
// global index first + i under key (k0, k1).  Writes theta[i][11].
cudaError_t launch_time_draw(const LikeConst& L, const DeviceBuffers& B, const float* ell, int n, long long first,
                             unsigned k0, unsigned k1, double* theta, cudaStream_t st);
cudaError_t launch_prior_transform(const PriorSlot* slots, int n_sampled, const double* u, int n, double* theta,
                                   cudaStream_t st, SkyFrame sky);
cudaError_t set_sweep_smem_limit(size_t bytes);

// Dynamic shared memory of the mixed sweep: data (float2 per detector and
// bin) plus the tile index of each bin of the slice.
inline size_t sweep_smem_bytes(int n_det, int slice_bins) {
  return (size_t)slice_bins * (n_det * sizeof(float2) + sizeof(int));
}

}  // namespace swig
