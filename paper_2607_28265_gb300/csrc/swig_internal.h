// Internal layout shared by the host side of libswig and its kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "swig.h"

namespace swig {

// Basis functions of the TaylorF2 intrinsic phase in cycles,
// P(f) = sum_j c_j phi_j(f)  (the v-power series of Psi_int/2pi rewritten in
// powers of f with theta-dependent coefficients).
enum Basis {
  B_M53 = 0,   // f^-5/3
  B_M1,        // f^-1
  B_M23,       // f^-2/3
  B_M13,       // f^-1/3
  B_LOG,       // ln f
  B_P13,       // f^1/3
  B_P13LOG,    // f^1/3 ln f
  B_P23,       // f^2/3
  B_P53,       // f^5/3
  B_P73,       // f^7/3
  B_ONE,       // 1
  NBASIS
};

constexpr int kTaylorDeg = 6;        // a_2 .. a_6 per tile
constexpr int kNumPoly = kTaylorDeg - 1;
constexpr int kChunk = 32;           // bins per warp step; tiles are multiples
constexpr int kMaxTileBins = 2048;
constexpr int kSweepThreads = 1024;  // 8 warp-groups of 4 warps
constexpr int kWarpGroups = kSweepThreads / 128;
constexpr int kPartialStride = 8;    // floats/doubles per (theta, slice) partial
constexpr int kAnchorStride = 12;    // floats per (theta, tile): A0, s_hi, s_lo, a2..a6, A_det[4]

// Per-tile table of basis values at the tile anchor f_a (first bin):
//   val   phi_j(f_a) as double-float (hi, lo)
//   slope phi_j'(f_a) * df as double-float
//   poly  phi_j^(n)(f_a) (df T)^n / n!, n = 2..kTaylorDeg, float
struct TileBasis {
  float val_hi[NBASIS], val_lo[NBASIS];
  float slope_hi[NBASIS], slope_lo[NBASIS];
  float poly[kNumPoly][NBASIS];
};

struct TileInfo {
  int k0;            // first bin (0-based within the grid)
  int nbins;         // bins in the tile (multiple of 32 except the grid's last)
  float fa_hi, fa_lo;  // anchor frequency f_a as double-float
  float inv_T;       // 1 / T, T = power-of-two tile span scaling the polynomial variable
  int split_bits;    // low mantissa bits cleared in the slope so x * slope_hi is exact
};

// Per-theta record written by the setup kernel (FP64 arithmetic).
struct EvalRecord {
  double c[NBASIS];              // intrinsic phase coefficients [cycles]
  float c_hi[NBASIS], c_lo[NBASIS];  // same as double-float
  double tau[SWIG_MAX_DET];      // t_c + geocentric delay [s]
  float tau_hi[SWIG_MAX_DET], tau_lo[SWIG_MAX_DET];
  double cre[SWIG_MAX_DET], cim[SWIG_MAX_DET];  // C_i (see loglike epilogue)
  double pre[SWIG_MAX_DET], pim[SWIG_MAX_DET];  // projection P_i, C_i = amp P_i
  double amp;                    // A(Mc) / d_L
  double mterm[8];               // cached mass factors (eta, dm, m1, m2, A, r, ir, ln pi M)
  double hh;                     // sum_i |C_i|^2 K_i
  double gdel[SWIG_MAX_DET];     // geocentric delay of each detector [s] (tau_i - t_c)
  int valid;
  int pad;
};

constexpr int kGaussLegendre = 64;  // nodes of the distance integral
constexpr int kMaxTmNodes = 65536;  // largest time-marginalisation grid

struct LikeConst {
  int n_det;
  int n_bins;
  int k_min;
  int n_tiles;
  int n_slices;
  int phase_marg;
  int fast_epilogue;  // mixed precision: log(i0e) of the phase marginal in FP32
  double df;
  double gmst;
  double K[SWIG_MAX_DET];        // 4 df sum f^-7/3 / S
  double DD;                     // sum_i <d_i|d_i>
  double inv_scale[SWIG_MAX_DET];  // data scale folded into C_i
  // FP32-friendly constants for projection-only evaluations:
  // amp_s = inv_scale * A1, amp_k = K * A1^2 with A1 the SPA amplitude of
  // Mc = 1 Msun at 1 Mpc, so C_i kappa_i and |C_i|^2 K_i stay O(1..1e6).
  float amp_s[SWIG_MAX_DET];
  float amp_k[SWIG_MAX_DET];
  double amp1;  // A1 itself
  double dten[SWIG_MAX_DET][6];  // detector tensor xx xy xz yy yz zz
  double vertex[SWIG_MAX_DET][3];
  // distance marginalisation (d_L slot marginalised): prior family and range,
  // Gauss-Legendre nodes and weights on [-1, 1]
  int dist_marg;
  int d_kind;
  double d_lo, d_hi;
  double gl_x[kGaussLegendre], gl_w[kGaussLegendre];
  // time marginalisation (t_c marginalised, heterodyned likelihood): tm_n
  // midpoint nodes t_j = tm_lo + (j + 1/2) tm_dt over the uniform t_c prior;
  // templates are built at t_c = tm_tref (the fiducial's) and shifted by
  // tm_t0 + j tm_dt = t_j - tm_tref
  int tm_n;
  double tm_lo, tm_dt, tm_tref, tm_t0;
  // non-uniform FFT form of the time pass (tm_M > 0): grid size, the node j0
  // of the reference shift tm_dref = tm_t0 + j0 tm_dt
  int tm_M, tm_j0;
  double tm_dref;
  // the gather's pieces (runs of at most 32 entries of one grid point) and
  // the grid points with entries
  int tm_pieces, tm_points;
  // heterodyned likelihood: 1 / |C0_i|^2 of the fiducial's projection factors
  double het_fid_iden[SWIG_MAX_DET];
};

}  // namespace swig
