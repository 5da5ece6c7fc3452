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
  const float* edge_basis;    // [2 * NBASIS][N_b + 1] phi_j(f_e): row 2j hi parts, row 2j+1 lo parts
  const float* edge_f;        // [2][N_b + 1] f_e: hi parts, lo parts
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

// Per-evaluation constants: coefficient and delay differences from the
// fiducial in double-float, and rho_i = C_i / C0_i.
template <int NDET>
struct HetPrep {
  dfl dc[NBASIS];
  dfl dtau[NDET];
  float rho_re[NDET], rho_im[NDET];
};

template <int NDET>
__device__ inline void het_prepare(const HetTables& H, const EvalRecord& r, HetPrep<NDET>& p) {
  const EvalRecord& f0 = *H.fid;
#pragma unroll
  for (int j = 0; j < NBASIS; ++j) p.dc[j] = df_from_double(r.c[j] - f0.c[j]);
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
    p.dtau[i] = df_from_double(r.tau[i] - f0.tau[i]);
    const double den = f0.cre[i] * f0.cre[i] + f0.cim[i] * f0.cim[i];
    p.rho_re[i] = (float)((r.cre[i] * f0.cre[i] + r.cim[i] * f0.cim[i]) / den);
    p.rho_im[i] = (float)((r.cim[i] * f0.cre[i] - r.cre[i] * f0.cim[i]) / den);
  }
}

// Bins [base, base + 31) of the contraction, accumulated into the lane's
// per-detector sums: lane l holds edge base + l, bin base + l uses edges l and
// l + 1 (the next edge by a shuffle).  All 32 lanes must call it together.
template <int NDET>
__device__ inline void het_chunk(const HetTables& H, const HetPrep<NDET>& p, int base, int lane, float* zr, float* zi,
                                 float* hh) {
  const float twopi = 6.283185307179586f;
  const int e = base + lane;
  float er[NDET], ei[NDET];
  if (e <= H.n_bins) {
    const size_t ne = (size_t)H.n_bins + 1;  // edges; lanes read consecutive edges of each row
    dfl dp = {0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < NBASIS; ++j)
      dp = df_add(dp, df_mul(p.dc[j], dfl{H.edge_basis[2 * j * ne + e], H.edge_basis[(2 * j + 1) * ne + e]}));
    const dfl fe = {H.edge_f[e], H.edge_f[ne + e]};
#pragma unroll
    for (int i = 0; i < NDET; ++i) {
      const float ph = df_frac(df_add(dp, df_mul(fe, p.dtau[i])));
      float s, co;
      __sincosf(twopi * ph, &s, &co);  // exp(-2 pi i ph) = co - i s
      er[i] = p.rho_re[i] * co + p.rho_im[i] * s;
      ei[i] = p.rho_im[i] * co - p.rho_re[i] * s;
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

// Warp-sum of the lane sums (all lanes receive them).
template <int NDET>
__device__ inline void het_warp_reduce(float* zr, float* zi, float* hh) {
#pragma unroll
  for (int i = 0; i < NDET; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      zr[i] += __shfl_xor_sync(0xffffffffu, zr[i], o);
      zi[i] += __shfl_xor_sync(0xffffffffu, zi[i], o);
      hh[i] += __shfl_xor_sync(0xffffffffu, hh[i], o);
    }
}

// FP64 epilogue: plain Re Z or phase-marginalised log I0(|Z|), minus
// <h|h>/2 and <d|d>/2.
__device__ inline double het_epilogue(const LikeConst& L, double Z_re, double Z_im, double HH) {
  const double base_ll = -0.5 * HH - 0.5 * L.DD;
  if (L.phase_marg) {
    const double x = sqrt(Z_re * Z_re + Z_im * Z_im);
    return (L.fast_epilogue ? x + (double)log_i0e_f32((float)x) : log_bessel_i0(x)) + base_ll;
  }
  return Z_re + base_ll;
}

__host__ __device__ inline int het_chunks(int n_bins) { return (n_bins + 30) / 31; }

// Per-detector sums cached for projection-only evaluations: (Z_i / C_i) /
// inv_scale_i as the chain's kappa, and <h|h>_i / |C_i|^2 times A1^2 (the
// heterodyned Z_i is linear and <h|h>_i quadratic in C_i).
__device__ inline void het_cache(const LikeConst& L, const EvalRecord& r, int i, double zr, double zi, double hh,
                                 double* kap2, double* vv) {
  const double cr = r.cre[i], ci = r.cim[i], c2 = cr * cr + ci * ci;
  if (c2 > 0.0) {
    kap2[0] = (zr * cr + zi * ci) / c2 / L.inv_scale[i];
    kap2[1] = (zi * cr - zr * ci) / c2 / L.inv_scale[i];
    *vv = hh / c2 * L.amp1 * L.amp1;
  } else {
    kap2[0] = kap2[1] = 0.0;
    *vv = 0.0;
  }
}

// One warp evaluates the heterodyned logL of record r (all lanes return it);
// optionally the per-detector cache of het_cache (lane 0 writes it).
template <int NDET>
__device__ inline double het_loglike_warp(const LikeConst& L, const HetTables& H, const EvalRecord& r, int lane,
                                          double* kap_out = nullptr, double* vv_out = nullptr) {
  if (!r.valid) {
    if (lane == 0 && kap_out)
      for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) kap_out[j] = 0.0;
    if (lane == 0 && vv_out)
      for (int i = 0; i < SWIG_MAX_DET; ++i) vv_out[i] = 0.0;
    return -INFINITY;
  }
  HetPrep<NDET> p;
  het_prepare<NDET>(H, r, p);
  float zr[NDET], zi[NDET], hh[NDET];
#pragma unroll
  for (int i = 0; i < NDET; ++i) zr[i] = zi[i] = hh[i] = 0.0f;
  const int nc = het_chunks(H.n_bins);
  for (int q = 0; q < nc; ++q) het_chunk<NDET>(H, p, 31 * q, lane, zr, zi, hh);
  het_warp_reduce<NDET>(zr, zi, hh);
  double Z_re = 0.0, Z_im = 0.0, HH = 0.0;
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
    Z_re += (double)zr[i];
    Z_im += (double)zi[i];
    HH += (double)hh[i];
  }
  if (lane == 0 && kap_out && vv_out) {
    for (int i = 0; i < SWIG_MAX_DET; ++i) {
      kap_out[2 * i] = kap_out[2 * i + 1] = 0.0;
      vv_out[i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < NDET; ++i) het_cache(L, r, i, zr[i], zi[i], hh[i], kap_out + 2 * i, vv_out + i);
  }
  return het_epilogue(L, Z_re, Z_im, HH);
}

}  // namespace swig
