// Device helpers for libswig: double-float arithmetic on the FP32 pipe, the
// TaylorF2 intrinsic-phase coefficients, detector projection and log I0.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "swig_internal.h"

namespace swig {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMtsunS = 4.925490947641266978e-6;  // G M_sun / c^3 [s]
constexpr double kCSI = 299792458.0;
constexpr double kMpcM = 3.0856775814913673e22;
constexpr double kEulerGamma = 0.57721566490153286061;

// ---------------------------------------------------------------------------
// Double-float ("float-float") arithmetic.  A value is hi + lo with
// |lo| <= ulp(hi)/2; the error-free transforms use round-to-nearest intrinsics
// so that no multiply-add contraction can alter them (Dekker 1971; Knuth
// TAOCP vol. 2, 4.2.2).  GB300 issues FP64 at ~1/64 of the FP32 rate, so the
// ~48-bit phase anchors are carried in pairs of floats instead.
// ---------------------------------------------------------------------------
struct dfl {
  float hi, lo;
};

// Philox-4x32-10 (Salmon, Moraes, Dror & Shaw 2011): 10 rounds of two 32x32
// multiplications with the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ dfl two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

// (a.hi + a.lo) * (b.hi + b.lo) to ~2^-46 relative.
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  dfl s = two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}

// Fractional part (nearest-integer reduction) of a double-float, returned as
// a float in [-0.5, 0.5] plus rounding of the low word.
__device__ __forceinline__ float df_frac(dfl a) {
  float n = rintf(a.hi);
  return __fadd_rn(__fsub_rn(a.hi, n), a.lo);  // a.hi - n is exact
}

// Round to the nearest integer on the FP32 add pipe: adding and subtracting
// 1.5 * 2^23 leaves the nearest integer for |v| < 2^22 (ties to even, as
// rintf), without occupying the SFU/conversion pipe that the sine and cosine
// need.
__device__ __forceinline__ float round_nearest(float v) {
  return __fsub_rn(__fadd_rn(v, 12582912.0f), 12582912.0f);
}

__device__ __forceinline__ dfl df_from_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return {h, l};
}

// ---------------------------------------------------------------------------
// TaylorF2 intrinsic phase in cycles as sum_j c_j phi_j(f) (basis in
// swig_internal.h).  Psi_int(f) = -pi/4 + 3/(128 eta v^5) sum_k alpha_k v^k
// with v = (pi M f)^(1/3); non-spinning alpha_k of Buonanno et al. 2009
// (PRD 80 084043, Eq. 3.18), aligned-spin 1.5PN spin-orbit and 2PN spin-spin
// terms (Poisson & Will 1995), tidal 5PN/6PN terms (Wade et al. 2014).
// ---------------------------------------------------------------------------
// Shared mass-dependent factors of the basis coefficients, computed once per
// (Mc, q): two reciprocals and three transcendentals on the critical path.
struct MassTerms {
  double eta, dm, m1, m2, A, r, ir, lpm;
};

__host__ __device__ inline MassTerms taylorf2_mass_terms(double mc, double q) {
  MassTerms t;
  const double opq = 1.0 + q;
  const double inv_opq = 1.0 / opq, inv_q = 1.0 / q;
  t.m1 = inv_opq;
  t.m2 = q * inv_opq;
  t.dm = (1.0 - q) * inv_opq;                 // (m1 - m2) / M
  t.eta = t.m1 * t.m2;                        // q / (1 + q)^2
  const double inv_eta = opq * opq * inv_q;   // 1 / eta
  t.A = (3.0 / (256.0 * kPi)) * inv_eta;      // 3 / (128 eta) in cycles
  // ln(pi M) = ln(pi T_sun Mc) - (3/5) ln eta = ln((pi T_sun Mc)^5 / eta^3) / 5
  // (one logarithm);  r = (pi M)^(1/3)
  const double x = kPi * kMtsunS * mc, x2 = x * x;
  t.lpm = 0.2 * log(x2 * x2 * x * (inv_eta * inv_eta * inv_eta));
  t.r = exp(t.lpm * (1.0 / 3.0));
  t.ir = 1.0 / t.r;
  return t;
}

// Spin terms: 1.5PN spin-orbit beta and 2PN spin-spin sigma enter alpha_3, alpha_4.
__host__ __device__ inline void taylorf2_spin_coeffs(const MassTerms& t, double chi1, double chi2, double* c) {
  const double eta = t.eta, eta2 = eta * eta;
  const double so = (113.0 / 12.0 * t.m1 * t.m1 + 6.25 * eta) * chi1 + (113.0 / 12.0 * t.m2 * t.m2 + 6.25 * eta) * chi2;
  const double ss = 79.0 / 8.0 * eta * chi1 * chi2;
  const double a3 = -16.0 * kPi + 4.0 * so;
  const double a4 = 15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta2 - 10.0 * ss;
  const double ir2 = t.ir * t.ir;
  c[B_M23] = t.A * a3 * ir2;
  c[B_M13] = t.A * a4 * t.ir;
}

// Tidal terms (Wade et al. 2014): 5PN and 6PN, alpha_10 and alpha_12.
__host__ __device__ inline void taylorf2_tidal_coeffs(const MassTerms& t, double lam1, double lam2, double* c) {
  const double eta = t.eta, eta2 = eta * eta, eta3 = eta2 * eta, dm = t.dm;
  const double lsum = lam1 + lam2, ldif = lam1 - lam2;
  const double lt = 8.0 / 13.0 * ((1.0 + 7.0 * eta - 31.0 * eta2) * lsum + dm * (1.0 + 9.0 * eta - 11.0 * eta2) * ldif);
  const double dlt = 0.5 * (dm * (1.0 - 13272.0 / 1319.0 * eta + 8944.0 / 1319.0 * eta2) * lsum +
                            (1.0 - 15910.0 / 1319.0 * eta + 32850.0 / 1319.0 * eta2 + 3380.0 / 1319.0 * eta3) * ldif);
  const double a10 = -19.5 * lt;
  const double a12 = -3115.0 / 64.0 * lt + 6595.0 / 364.0 * dm * dlt;
  const double r2 = t.r * t.r, r5 = r2 * r2 * t.r, r7 = r5 * r2;
  c[B_P53] = t.A * a10 * r5;
  c[B_P73] = t.A * a12 * r7;
}

__host__ __device__ inline void taylorf2_basis_coeffs_from(const MassTerms& t, double chi1, double chi2,
                                                           double lam1, double lam2, double* c) {
  const double eta = t.eta, eta2 = eta * eta, eta3 = eta2 * eta;
  const double pi2 = kPi * kPi;
  const double a0 = 1.0;
  const double a2 = 3715.0 / 756.0 + 55.0 / 9.0 * eta;
  const double a5 = kPi * (38645.0 / 756.0 - 65.0 / 9.0 * eta);
  const double a5log = 3.0 * a5;
  const double a6 = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi2 - 6848.0 / 21.0 * kEulerGamma +
                    (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi2) * eta + 76055.0 / 1728.0 * eta2 -
                    127825.0 / 1296.0 * eta3;
  const double a6log = -6848.0 / 21.0;
  const double a7 = kPi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta2);
  const double ir2 = t.ir * t.ir, ir3 = ir2 * t.ir, ir5 = ir3 * ir2;
  const double r2 = t.r * t.r;
  const double third = 1.0 / 3.0;
  const double ln4 = 1.3862943611198906188, ln_vlso = -0.89587973461402746;  // ln 4, -ln(6)/2
  c[B_M53] = t.A * a0 * ir5;
  c[B_M1] = t.A * a2 * ir3;
  c[B_LOG] = t.A * a5log * third;
  c[B_P13] = t.A * t.r * (a6 + a6log * (ln4 + t.lpm * third));
  c[B_P13LOG] = t.A * t.r * a6log * third;
  c[B_P23] = t.A * a7 * r2;
  c[B_ONE] = t.A * (a5 + a5log * (t.lpm * third - ln_vlso)) - 0.125;
  taylorf2_spin_coeffs(t, chi1, chi2, c);
  taylorf2_tidal_coeffs(t, lam1, lam2, c);
}

__host__ __device__ inline void taylorf2_basis_coeffs(double mc, double q, double chi1, double chi2,
                                                      double lam1, double lam2, double* c) {
  taylorf2_basis_coeffs_from(taylorf2_mass_terms(mc, q), chi1, chi2, lam1, lam2, c);
}

// sqrt(5/24) pi^(-2/3) (G Mc / c^3)^(5/6) c / (1 Mpc): Newtonian SPA amplitude
// times d_L[Mpc].
__host__ __device__ inline double amplitude_per_mpc(double mc) {
  return sqrt(5.0 / 24.0) * exp(-2.0 / 3.0 * log(kPi)) * exp(5.0 / 6.0 * log(mc * kMtsunS)) * kCSI / kMpcM;
}

// Antenna patterns of detector tensor D (xx xy xz yy yz zz) for a source at
// (ra, dec), polarisation psi, Greenwich sidereal time gmst; polarisation
// basis X = -cos(psi) e_east + sin(psi) e_north, Y = sin(psi) e_east +
// cos(psi) e_north at the source direction.
__device__ inline void antenna_fp_fx(const double* d, double ra, double dec, double psi, double gmst,
                                     double* fp, double* fx) {
  double sl, cl, sd, cd, sp, cp;
  sincos(ra - gmst, &sl, &cl);
  sincos(dec, &sd, &cd);
  sincos(psi, &sp, &cp);
  const double east[3] = {-sl, cl, 0.0};
  const double north[3] = {-sd * cl, -sd * sl, cd};
  double X[3], Y[3];
  for (int k = 0; k < 3; ++k) {
    X[k] = -cp * east[k] + sp * north[k];
    Y[k] = sp * east[k] + cp * north[k];
  }
  // quadratic forms a^T D b with D symmetric
  auto form = [d](const double* a, const double* b) {
    return a[0] * (d[0] * b[0] + d[1] * b[1] + d[2] * b[2]) + a[1] * (d[1] * b[0] + d[3] * b[1] + d[4] * b[2]) +
           a[2] * (d[2] * b[0] + d[4] * b[1] + d[5] * b[2]);
  };
  *fp = form(X, X) - form(Y, Y);
  *fx = 2.0 * form(X, Y);
}

// Arrival time at a detector minus arrival at Earth's centre: -n.r / c.
__device__ inline double geocentric_delay(const double* vertex, double ra, double dec, double gmst) {
  double sl, cl, sd, cd;
  sincos(ra - gmst, &sl, &cl);
  sincos(dec, &sd, &cd);
  return -(cd * cl * vertex[0] + cd * sl * vertex[1] + sd * vertex[2]) / kCSI;
}

// log I0(x) for x >= 0: power series sum_k (x^2/4)^k / (k!)^2 below 20, and
// the large-argument expansion I0(x) ~ e^x / sqrt(2 pi x) sum_k ((2k-1)!!)^2 /
// (k! (8x)^k) above (Abramowitz & Stegun 9.6.10, 9.7.1).  The series terms
// use precomputed ratios (no division in the large-argument loop).
__host__ __device__ inline double log_bessel_i0(double x) {
  if (x < 20.0) {
    const double y = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 200; ++k) {  // rare: only for |Z| < 20
      term *= y / ((double)k * (double)k);
      sum += term;
      if (term < 1e-17 * sum) break;
    }
    return log(sum);
  }
  const double t = 0.125 / x;
  // ((2k-1)^2 / k) for k = 1..12
  const double r[12] = {1.0, 4.5, 25.0 / 3.0, 12.25, 16.2, 121.0 / 6.0, 169.0 / 7.0, 28.125,
                        289.0 / 9.0, 36.1, 441.0 / 11.0, 529.0 / 12.0};
  double term = 1.0, sum = 1.0;
  for (int k = 0; k < 12; ++k) {
    term *= r[k] * t;
    sum += term;
  }
  return x - 0.5 * log(2.0 * kPi * x) + log(sum);
}

// ---------------------------------------------------------------------------
// Per-theta setup (FP64): phase coefficients, delays, complex projection
// factors C_i = amp P_i so that h_i(f) = C_i f^(-7/6) exp(-2 pi i (P(f) + f tau_i)),
// with amp = A(Mc) / d_L and P_i = [F+_i (1 + cos^2 i)/2 - i Fx_i cos i] e^{i phi_c}.
// The pieces are separate so that a Gibbs block recomputes only what it moves.
// ---------------------------------------------------------------------------
__device__ inline bool theta_valid(const double* th) {
  double s = 0.0;
  for (int j = 0; j < SWIG_N_PARAMS; ++j) s += th[j];
  return (th[0] > 0.0) && (th[1] > 0.0) && (th[1] <= 1.0) && (th[6] > 0.0) && isfinite(s);
}

// split = false leaves c_hi / c_lo to the caller (a warp splits the
// coefficients one per lane).
__device__ inline void setup_intrinsic(const double* th, EvalRecord* rec, bool split = true) {
  double c[NBASIS];
  if (rec->valid) {
    const MassTerms t = taylorf2_mass_terms(th[0], th[1]);
    taylorf2_basis_coeffs_from(t, th[2], th[3], th[4], th[5], c);
    rec->mterm[0] = t.eta;
    rec->mterm[1] = t.dm;
    rec->mterm[2] = t.m1;
    rec->mterm[3] = t.m2;
    rec->mterm[4] = t.A;
    rec->mterm[5] = t.r;
    rec->mterm[6] = t.ir;
    rec->mterm[7] = t.lpm;
  } else {
    for (int j = 0; j < NBASIS; ++j) c[j] = 0.0;
  }
  for (int j = 0; j < NBASIS; ++j) {
    rec->c[j] = c[j];
    if (split) {
      dfl v = df_from_double(c[j]);
      rec->c_hi[j] = v.hi;
      rec->c_lo[j] = v.lo;
    }
  }
}

// Only the spin (slots 2, 3) or only the tidal (slots 4, 5) coefficients.
__device__ inline void setup_intrinsic_partial(const double* th, EvalRecord* rec, bool spin, bool tide,
                                               bool split = true) {
  if (!rec->valid) return;
  MassTerms t;  // Mc and q are unchanged: reuse the cached mass factors
  t.eta = rec->mterm[0];
  t.dm = rec->mterm[1];
  t.m1 = rec->mterm[2];
  t.m2 = rec->mterm[3];
  t.A = rec->mterm[4];
  t.r = rec->mterm[5];
  t.ir = rec->mterm[6];
  t.lpm = rec->mterm[7];
  double c[NBASIS];
  for (int j = 0; j < NBASIS; ++j) c[j] = rec->c[j];
  if (spin) taylorf2_spin_coeffs(t, th[2], th[3], c);
  if (tide) taylorf2_tidal_coeffs(t, th[4], th[5], c);
  const int js[4] = {B_M23, B_M13, B_P53, B_P73};
  for (int q = 0; q < 4; ++q) {
    const int j = js[q];
    rec->c[j] = c[j];
    if (split) {
      dfl v = df_from_double(c[j]);
      rec->c_hi[j] = v.hi;
      rec->c_lo[j] = v.lo;
    }
  }
}

__device__ inline void setup_amp(const double* th, EvalRecord* rec) {
  rec->amp = rec->valid ? amplitude_per_mpc(th[0]) / th[6] : 0.0;
}

__device__ inline void setup_projection(const LikeConst& L, const double* th, EvalRecord* rec) {
  const double ci = cos(th[7]);
  const double plus = 0.5 * (1.0 + ci * ci), cross = -ci;  // h+ ~ plus, hx ~ i*cross
  double sph = 0.0, cph = 1.0;
  if (!L.phase_marg) sincos(th[12], &sph, &cph);
  for (int i = 0; i < SWIG_MAX_DET; ++i) {
    if (i >= L.n_det) {
      rec->pre[i] = rec->pim[i] = 0.0;
      continue;
    }
    double fp, fx;
    antenna_fp_fx(L.dten[i], th[9], th[10], th[8], L.gmst, &fp, &fx);
    const double re0 = fp * plus, im0 = fx * cross;
    rec->pre[i] = re0 * cph - im0 * sph;
    rec->pim[i] = re0 * sph + im0 * cph;
  }
}

// FP32 variants for the mixed-precision sampler: C_i is needed to ~1e-7
// relative (its error enters logL as ~1e-7 |C kappa|), far below the tolerance.
__device__ inline void setup_amp_f32(const double* th, EvalRecord* rec) {
  const float rel = exp2f(0.8333333333f * log2f((float)th[0])) / (float)th[6];
  rec->amp = rec->valid ? (double)rel * amplitude_per_mpc(1.0) : 0.0;
}

__device__ inline void setup_projection_f32(const LikeConst& L, const double* th, EvalRecord* rec) {
  float sl, cl, sd, cd, sp, cp;
  sincosf((float)(th[9] - L.gmst), &sl, &cl);
  sincosf((float)th[10], &sd, &cd);
  sincosf((float)th[8], &sp, &cp);
  const float east[3] = {-sl, cl, 0.0f};
  const float north[3] = {-sd * cl, -sd * sl, cd};
  float X[3], Y[3];
  for (int k = 0; k < 3; ++k) {
    X[k] = -cp * east[k] + sp * north[k];
    Y[k] = sp * east[k] + cp * north[k];
  }
  const float ci = cosf((float)th[7]);
  const float plus = 0.5f * (1.0f + ci * ci), cross = -ci;
  float sph = 0.0f, cph = 1.0f;
  if (!L.phase_marg) sincosf((float)th[12], &sph, &cph);
  for (int i = 0; i < SWIG_MAX_DET; ++i) {
    if (i >= L.n_det) {
      rec->pre[i] = rec->pim[i] = 0.0;
      continue;
    }
    float d[6];
    for (int q = 0; q < 6; ++q) d[q] = (float)L.dten[i][q];
    auto form = [&d](const float* a, const float* b) {
      return a[0] * (d[0] * b[0] + d[1] * b[1] + d[2] * b[2]) + a[1] * (d[1] * b[0] + d[3] * b[1] + d[4] * b[2]) +
             a[2] * (d[2] * b[0] + d[4] * b[1] + d[5] * b[2]);
    };
    const float fp = form(X, X) - form(Y, Y), fx = 2.0f * form(X, Y);
    const float re0 = fp * plus, im0 = fx * cross;
    rec->pre[i] = (double)(re0 * cph - im0 * sph);
    rec->pim[i] = (double)(re0 * sph + im0 * cph);
  }
}

__device__ inline void setup_delays(const LikeConst& L, const double* th, EvalRecord* rec) {
  double sl, cl, sd, cd;
  sincos(th[9] - L.gmst, &sl, &cl);
  sincos(th[10], &sd, &cd);
  const double n0 = cd * cl * (-1.0 / kCSI), n1 = cd * sl * (-1.0 / kCSI), n2 = sd * (-1.0 / kCSI);
  for (int i = 0; i < SWIG_MAX_DET; ++i) {
    const double gd = i < L.n_det ? (n0 * L.vertex[i][0] + n1 * L.vertex[i][1] + n2 * L.vertex[i][2]) : 0.0;
    const double tau = i < L.n_det ? th[11] + gd : 0.0;
    rec->gdel[i] = gd;
    rec->tau[i] = tau;
    dfl tv = df_from_double(tau);
    rec->tau_hi[i] = tv.hi;
    rec->tau_lo[i] = tv.lo;
  }
}

// One detector's share of setup_projection(_f32) and setup_delays, so that a
// warp can set up a record with one lane per piece (setup_record_warp).
__device__ inline void setup_projection_det(const LikeConst& L, const double* th, int i, bool f32, EvalRecord* rec) {
  if (f32) {
    float sl, cl, sd, cd, sp, cp;
    sincosf((float)(th[9] - L.gmst), &sl, &cl);
    sincosf((float)th[10], &sd, &cd);
    sincosf((float)th[8], &sp, &cp);
    const float east[3] = {-sl, cl, 0.0f};
    const float north[3] = {-sd * cl, -sd * sl, cd};
    float X[3], Y[3];
    for (int k = 0; k < 3; ++k) {
      X[k] = -cp * east[k] + sp * north[k];
      Y[k] = sp * east[k] + cp * north[k];
    }
    const float ci = cosf((float)th[7]);
    const float plus = 0.5f * (1.0f + ci * ci), cross = -ci;
    float sph = 0.0f, cph = 1.0f;
    if (!L.phase_marg) sincosf((float)th[12], &sph, &cph);
    float d[6];
    for (int q = 0; q < 6; ++q) d[q] = (float)L.dten[i][q];
    auto form = [&d](const float* a, const float* b) {
      return a[0] * (d[0] * b[0] + d[1] * b[1] + d[2] * b[2]) + a[1] * (d[1] * b[0] + d[3] * b[1] + d[4] * b[2]) +
             a[2] * (d[2] * b[0] + d[4] * b[1] + d[5] * b[2]);
    };
    const float fp = form(X, X) - form(Y, Y), fx = 2.0f * form(X, Y);
    const float re0 = fp * plus, im0 = fx * cross;
    rec->pre[i] = (double)(re0 * cph - im0 * sph);
    rec->pim[i] = (double)(re0 * sph + im0 * cph);
  } else {
    const double ci = cos(th[7]);
    const double plus = 0.5 * (1.0 + ci * ci), cross = -ci;
    double sph = 0.0, cph = 1.0;
    if (!L.phase_marg) sincos(th[12], &sph, &cph);
    double fp, fx;
    antenna_fp_fx(L.dten[i], th[9], th[10], th[8], L.gmst, &fp, &fx);
    const double re0 = fp * plus, im0 = fx * cross;
    rec->pre[i] = re0 * cph - im0 * sph;
    rec->pim[i] = re0 * sph + im0 * cph;
  }
}

// Detector i's delay from the sines and cosines of (RA - GMST) and Dec.
__device__ inline void setup_delay_det_sc(const LikeConst& L, const double* th, int i, double sl, double cl,
                                          double sd, double cd, EvalRecord* rec) {
  const double n0 = cd * cl * (-1.0 / kCSI), n1 = cd * sl * (-1.0 / kCSI), n2 = sd * (-1.0 / kCSI);
  const double gd = (n0 * L.vertex[i][0] + n1 * L.vertex[i][1] + n2 * L.vertex[i][2]);
  const double tau = th[11] + gd;
  rec->gdel[i] = gd;
  rec->tau[i] = tau;
  dfl tv = df_from_double(tau);
  rec->tau_hi[i] = tv.hi;
  rec->tau_lo[i] = tv.lo;
}

__device__ inline void setup_delay_det(const LikeConst& L, const double* th, int i, EvalRecord* rec) {
  double sl, cl, sd, cd;
  sincos(th[9] - L.gmst, &sl, &cl);
  sincos(th[10], &sd, &cd);
  setup_delay_det_sc(L, th, i, sl, cl, sd, cd, rec);
}

// A move of t_c alone: the record's geocentric delay of detector i is kept,
// tau_i = t_c + gdel_i (the same sum setup_delay_det forms).
__device__ inline void setup_tc_det(const double* th, int i, EvalRecord* rec) {
  const double tau = th[11] + rec->gdel[i];
  rec->tau[i] = tau;
  dfl tv = df_from_double(tau);
  rec->tau_hi[i] = tv.hi;
  rec->tau_lo[i] = tv.lo;
}

__device__ inline void setup_combine(const LikeConst& L, EvalRecord* rec) {
  double hh = 0.0;
  for (int i = 0; i < SWIG_MAX_DET; ++i) {
    rec->cre[i] = rec->amp * rec->pre[i];
    rec->cim[i] = rec->amp * rec->pim[i];
    if (i < L.n_det) hh += (rec->cre[i] * rec->cre[i] + rec->cim[i] * rec->cim[i]) * L.K[i];
  }
  rec->hh = hh;
}

__device__ inline void setup_record(const LikeConst& L, const double* th, EvalRecord* rec) {
  rec->valid = theta_valid(th) ? 1 : 0;
  setup_intrinsic(th, rec);
  setup_amp(th, rec);
  setup_projection(L, th, rec);
  setup_delays(L, th, rec);
  setup_combine(L, rec);
}

// ---------------------------------------------------------------------------
// Distance marginalisation (Sec. 3.1).  With d_L marginalised the record is
// set up at d_L = 1 Mpc, where the template gives Z1 = sum_i C_i kappa_i and
// H1 = sum_i |C_i|^2 K_i; at distance d they scale as Z1/d and H1/d^2, so
//   log L_marg = log int pi(d) exp(Re Z1 / d - H1 / (2 d^2)) dd - <d|d>/2
// (log I0(|Z1| / d) in place of Re Z1 / d with phi_c marginalised).  The
// integral is taken over u = 1/d by 64-node Gauss-Legendre on a window of
// +-12 standard deviations (1 / sqrt(H1)) around the peak u* = max(X, 0) / H1
// (X = Re Z1 or |Z1|), cut to the prior, or 12 standard deviations from the
// nearer prior edge when the peak lies outside; the exponent is FP64, the
// slowly varying log-prior, Jacobian and log(i0e) terms FP32.
// ---------------------------------------------------------------------------
__host__ __device__ inline float log_i0e_f32(float x) {  // log(I0(x) e^-x), x >= 0
  if (x < 20.0f) {
    const float y = 0.25f * x * x;
    float term = 1.0f, sum = 1.0f;
    for (int k = 1; k < 64; ++k) {
      term *= y / (float)(k * k);
      sum += term;
      if (term < 1e-8f * sum) break;
    }
    return logf(sum) - x;
  }
  const float t = 1.0f / (8.0f * x);
  const float s = 1.0f + t * (1.0f + t * (4.5f + t * (37.5f + t * 459.375f)));
  return -0.5f * logf(6.283185307179586f * x) + logf(s);
}

// log of pi(1/u) / u^2 (prior density in d times the Jacobian |dd/du|).
__host__ __device__ inline float distance_log_density_u(const LikeConst& L, float u) {
  const float lu = logf(u);
  if (L.d_kind == SWIG_PRIOR_POWER2)  // pi(d) = 3 d^2 / (hi^3 - lo^3)
    return logf(3.0f / (float)(L.d_hi * L.d_hi * L.d_hi - L.d_lo * L.d_lo * L.d_lo)) - 4.0f * lu;
  return -logf((float)(L.d_hi - L.d_lo)) - 2.0f * lu;  // uniform
}

// Integration window in u = 1/d.
__host__ __device__ inline void distance_window(const LikeConst& L, double X, double H, double* lo, double* hi) {
  const double ua = 1.0 / L.d_hi, ub = 1.0 / L.d_lo;
  double a = ua, b = ub;
  if (H > 0.0) {  // (no template power: the integrand is the prior, take the whole range)
    const double us = fmax(X, 0.0) / H, su = 12.0 / sqrt(H);
    a = fmax(ua, us - su);
    b = fmin(ub, us + su);
    if (a >= b) {  // peak outside the prior: the window at the nearer edge
      if (us < ua) {
        a = ua;
        b = fmin(ub, ua + su);
      } else {
        a = fmax(ua, ub - su);
        b = ub;
      }
    }
  }
  *lo = a;
  *hi = b;
}

// Exponent of the integrand in u (FP64 part, without -<d|d>/2).
__host__ __device__ inline double distance_exponent(const LikeConst& L, double zre, double X, double H, double u) {
  const double core = L.phase_marg ? X * u + (double)log_i0e_f32((float)(X * u)) : zre * u;
  return core - 0.5 * H * u * u + (double)distance_log_density_u(L, (float)u);
}

__host__ __device__ inline double distance_marg_logl(const LikeConst& L, double zre, double zim, double H) {
  const double X = L.phase_marg ? sqrt(zre * zre + zim * zim) : zre;
  double a, b;
  distance_window(L, X, H, &a, &b);
  const double mid = 0.5 * (a + b), half = 0.5 * (b - a);
  double M = -INFINITY;
  for (int k = 0; k < kGaussLegendre; ++k) M = fmax(M, distance_exponent(L, zre, X, H, mid + half * L.gl_x[k]));
  double sum = 0.0;
  for (int k = 0; k < kGaussLegendre; ++k)
    sum += L.gl_w[k] * (double)expf((float)(distance_exponent(L, zre, X, H, mid + half * L.gl_x[k]) - M));
  return M + log(half * sum) - 0.5 * L.DD;
}

// logL from the per-detector sums kappa_i = sum_k D_i(k) exp(-2 pi i phi_i(k))
// (data scaled by 1/inv_scale_i): Eq. 2 expanded as
// sum_i Re(C_i kappa_i) - 1/2 sum_i |C_i|^2 K_i - 1/2 sum_i <d_i|d_i>, or with
// phi_c marginalised log I0(|sum_i C_i kappa_i|) - ...
__device__ inline double loglike_epilogue(const LikeConst& L, const EvalRecord& rec, const double* kre,
                                          const double* kim) {
  if (!rec.valid) return -INFINITY;
  double zr = 0.0, zi = 0.0;
  for (int i = 0; i < L.n_det; ++i) {
    const double a = kre[i] * L.inv_scale[i], b = kim[i] * L.inv_scale[i];
    zr += rec.cre[i] * a - rec.cim[i] * b;
    zi += rec.cre[i] * b + rec.cim[i] * a;
  }
  if (L.dist_marg) return distance_marg_logl(L, zr, zi, rec.hh);
  const double base = -0.5 * rec.hh - 0.5 * L.DD;
  if (L.phase_marg) {
    const double x = sqrt(zr * zr + zi * zi);
    // log I0(x) = x + log(i0e(x)); the second term is O(log x) and needs only
    // FP32 in the mixed-precision path (absolute error ~1e-6)
    return (L.fast_epilogue ? x + (double)log_i0e_f32((float)x) : log_bessel_i0(x)) + base;
  }
  return zr + base;
}

}  // namespace swig

#include "kernels.h"

namespace swig {

// Inverse CDFs of the Table I prior families on [lo, hi], with the slot's
// precomputed constants (c1, c2): sine p ~ sin x: x = acos(cos lo - u (cos lo -
// cos hi)); cosine p ~ cos x: x = asin(sin lo + u (sin hi - sin lo)); p ~ x^2:
// x = (lo^3 + u (hi^3 - lo^3))^(1/3); uniform: lo + u (hi - lo).
__host__ __device__ inline double prior_slot_inverse(const PriorSlot& s, double u) {
  switch (s.kind) {
    case SWIG_PRIOR_SINE:
      return acos(s.c1 - u * (s.c1 - s.c2));
    case SWIG_PRIOR_COSINE:
      return asin(s.c1 + u * (s.c2 - s.c1));
    case SWIG_PRIOR_POWER2:
      return cbrt(s.c1 + u * (s.c2 - s.c1));
    default:
      return s.lo + u * (s.hi - s.lo);
  }
}

// Same families with FP32 transcendentals (relative error ~1e-7 on theta):
// used by the mixed-precision sampler, where the likelihood is evaluated at
// exactly the returned theta, so only the prior measure moves by ~1e-7.
__device__ inline double prior_slot_inverse_f32(const PriorSlot& s, double u) {
  switch (s.kind) {
    case SWIG_PRIOR_SINE:
      return (double)acosf((float)(s.c1 - u * (s.c1 - s.c2)));
    case SWIG_PRIOR_COSINE:
      return (double)asinf((float)(s.c1 + u * (s.c2 - s.c1)));
    case SWIG_PRIOR_POWER2:
      return (double)cbrtf((float)(s.c1 + u * (s.c2 - s.c1)));
    default:
      return s.lo + u * (s.hi - s.lo);
  }
}

// Unit-cube coordinates of the sampled slots -> full 13-vector.
// (azimuth, zenith) about the frame's ez -> (RA, Dec): n = sin z cos a ex +
// sin z sin a ey + cos z ez in the Earth-fixed frame, Dec = asin n_z,
// RA = atan2(n_y, n_x) + GMST (mod 2 pi).
__host__ __device__ inline void sky_frame_to_radec(const SkyFrame& F, double az, double zen, double* ra,
                                                   double* dec) {
  double sa, ca, sz, cz;
  sa = sin(az);
  ca = cos(az);
  sz = sin(zen);
  cz = cos(zen);
  double n[3];
  for (int k = 0; k < 3; ++k) n[k] = sz * ca * F.ex[k] + sz * sa * F.ey[k] + cz * F.ez[k];
  *dec = asin(fmin(1.0, fmax(-1.0, n[2])));
  double r = atan2(n[1], n[0]) + F.gmst;
  r = fmod(r, 2.0 * kPi);
  if (r < 0.0) r += 2.0 * kPi;
  *ra = r;
}

__host__ __device__ inline void prior_map(const PriorSlot* slots, const double* u, double* th,
                                          const SkyFrame* sky = nullptr);

__host__ __device__ inline void prior_map(const PriorSlot* slots, const double* u, double* th, const SkyFrame* sky) {
  int j = 0;
  for (int i = 0; i < SWIG_N_PARAMS; ++i) {
    const PriorSlot& s = slots[i];
    if (s.mode == SWIG_MODE_FIXED) {
      th[i] = s.value;
    } else if (s.mode == SWIG_MODE_MARG) {
      th[i] = s.value;  // phi_c: 0; d_L: the 1 Mpc reference distance
    } else {
      th[i] = prior_slot_inverse(s, u[j++]);
    }
  }
  if (sky && sky->on) sky_frame_to_radec(*sky, th[9], th[10], &th[9], &th[10]);
}

}  // namespace swig

namespace swig {
inline PriorSlot make_prior_slot(int kind, int mode, double lo, double hi, double value) {
  PriorSlot s{kind, mode, lo, hi, value, 0.0, 0.0};
  if (kind == SWIG_PRIOR_SINE) {
    s.c1 = std::cos(lo);
    s.c2 = std::cos(hi);
  } else if (kind == SWIG_PRIOR_COSINE) {
    s.c1 = std::sin(lo);
    s.c2 = std::sin(hi);
  } else if (kind == SWIG_PRIOR_POWER2) {
    s.c1 = lo * lo * lo;
    s.c2 = hi * hi * hi;
  }
  return s;
}
}  // namespace swig
