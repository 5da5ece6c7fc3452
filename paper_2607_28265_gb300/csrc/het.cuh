// Heterodyned (relative-binning) likelihood (Sec. 3.4 of the paper) on the device.
//
// With the fiducial waveform h0 the ratio r_i(f) = h_i(f) / h0_i(f) is, for
// this model, (C_i / C0_i) exp(-2 pi i (dP(f) + f dtau_i)) with dP = P - P0 and
// dtau_i = tau_i - tau0_i (the f^-7/6 amplitude cancels).  It is evaluated at
// the N_b + 1 bin edges and taken linear inside each bin:
//   r0_b = (r(e_b) + r(e_b+1)) / 2,  r1_b = (r(e_b+1) - r(e_b)) / (e_b+1 - e_b),
//   Z_i  = sum_b A0_ib r0_b + A1_ib r1_b,
//   HH_i = sum_b B0_ib |r0_b|^2 + 2 B1_ib Re(r0_b conj(r1_b)),
// with the summary data A0, A1, B0, B1 (host FP64, stored FP32).  dP at an
// edge is a double-float sum of (c_j - c0_j) phi_j(f_e) (it can reach hundreds
// of cycles far from the fiducial); the contraction itself is FP32 per bin with
// a pairwise (warp-shuffle) reduction and an FP64 epilogue.
#pragma once

#include "device_common.cuh"

namespace swig {

struct HetTables {
  int n_bins;                 // N_b
  const float* edge_basis;    // [N_b + 1][2 * NBASIS] phi_j(f_e) as (hi, lo)
  const float* edge_f;        // [N_b + 1][2] f_e as (hi, lo)
  const float* inv_width;     // [N_b] 1 / (e_{b+1} - e_b)
  const float4* coef;         // [n_det][N_b] (A0.re, A0.im, A1.re, A1.im)
  const float2* coefB;        // [n_det][N_b] (B0, B1)
  const EvalRecord* fid;      // fiducial record
};

__host__ __device__ inline HetTables het_tables(const DeviceBuffers& B) {
  HetTables H;
  H.n_bins = B.het_nb;
  H.edge_basis = B.het_edge_basis;
  H.edge_f = B.het_edge_f;
  H.inv_width = B.het_inv_width;
  H.coef = B.het_coef;
  H.coefB = B.het_coefB;
  H.fid = B.het_fid;
  return H;
}

// One warp evaluates the heterodyned logL of record r (all lanes return it).
// z_out/hh_out (optional, lane-uniform): per-detector Z_i (re, im) and HH_i.
template <int NDET>
__device__ inline double het_loglike_warp(const LikeConst& L, const HetTables& H, const EvalRecord& r, int lane,
                                          double* z_out = nullptr, double* hh_out = nullptr) {
  if (!r.valid) return -INFINITY;
  const EvalRecord& f0 = *H.fid;
  // coefficient differences in double-float (uniform)
  dfl dc[NBASIS];
#pragma unroll
  for (int j = 0; j < NBASIS; ++j) dc[j] = df_from_double(r.c[j] - f0.c[j]);
  dfl dtau[NDET];
  float rho_re[NDET], rho_im[NDET];
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
    dtau[i] = df_from_double(r.tau[i] - f0.tau[i]);
    // rho = C_i / C0_i
    const double den = f0.cre[i] * f0.cre[i] + f0.cim[i] * f0.cim[i];
    rho_re[i] = (float)((r.cre[i] * f0.cre[i] + r.cim[i] * f0.cim[i]) / den);
    rho_im[i] = (float)((r.cim[i] * f0.cre[i] - r.cre[i] * f0.cim[i]) / den);
  }
  float zr[NDET], zi[NDET], hh[NDET];
#pragma unroll
  for (int i = 0; i < NDET; ++i) zr[i] = zi[i] = hh[i] = 0.0f;
  const float twopi = 6.283185307179586f;
  // chunks of 31 bins: lane l holds edge base + l; bin base + l uses edges l, l + 1
  for (int base = 0; base < H.n_bins; base += 31) {
    const int e = base + lane;
    float er[NDET], ei[NDET];
    if (e <= H.n_bins) {
      const float* eb = H.edge_basis + (size_t)e * 2 * NBASIS;
      dfl dp = {0.0f, 0.0f};
#pragma unroll
      for (int j = 0; j < NBASIS; ++j) dp = df_add(dp, df_mul(dc[j], dfl{eb[2 * j], eb[2 * j + 1]}));
      const dfl fe = {H.edge_f[2 * e], H.edge_f[2 * e + 1]};
#pragma unroll
      for (int i = 0; i < NDET; ++i) {
        const float ph = df_frac(df_add(dp, df_mul(fe, dtau[i])));
        float s, co;
        __sincosf(twopi * ph, &s, &co);  // exp(-2 pi i ph) = co - i s
        er[i] = rho_re[i] * co + rho_im[i] * s;
        ei[i] = rho_im[i] * co - rho_re[i] * s;
      }
    } else {
#pragma unroll
      for (int i = 0; i < NDET; ++i) er[i] = ei[i] = 0.0f;
    }
    const int b = base + lane;
    const bool has_bin = lane < 31 && b < H.n_bins;
    const float iw = has_bin ? H.inv_width[b] : 0.0f;
#pragma unroll
    for (int i = 0; i < NDET; ++i) {
      const float nr = __shfl_down_sync(0xffffffffu, er[i], 1);
      const float ni = __shfl_down_sync(0xffffffffu, ei[i], 1);
      if (has_bin) {
        const float r0r = 0.5f * (er[i] + nr), r0i = 0.5f * (ei[i] + ni);
        const float r1r = (nr - er[i]) * iw, r1i = (ni - ei[i]) * iw;
        const float4 a = H.coef[(size_t)i * H.n_bins + b];
        const float2 bb = H.coefB[(size_t)i * H.n_bins + b];
        zr[i] += a.x * r0r - a.y * r0i + a.z * r1r - a.w * r1i;
        zi[i] += a.x * r0i + a.y * r0r + a.z * r1i + a.w * r1r;
        hh[i] += bb.x * (r0r * r0r + r0i * r0i) + 2.0f * bb.y * (r0r * r1r + r0i * r1i);
      }
    }
  }
  double Z_re = 0.0, Z_im = 0.0, HH = 0.0;
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      zr[i] += __shfl_xor_sync(0xffffffffu, zr[i], o);
      zi[i] += __shfl_xor_sync(0xffffffffu, zi[i], o);
      hh[i] += __shfl_xor_sync(0xffffffffu, hh[i], o);
    }
    Z_re += (double)zr[i];
    Z_im += (double)zi[i];
    HH += (double)hh[i];
    if (z_out) {
      z_out[2 * i] = zr[i];
      z_out[2 * i + 1] = zi[i];
    }
    if (hh_out) hh_out[i] = hh[i];
  }
  const double base_ll = -0.5 * HH - 0.5 * L.DD;
  if (L.phase_marg) return log_bessel_i0(sqrt(Z_re * Z_re + Z_im * Z_im)) + base_ll;
  return Z_re + base_ll;
}

}  // namespace swig
