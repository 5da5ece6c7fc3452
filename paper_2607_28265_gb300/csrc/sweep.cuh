// Bin-sweep device code shared by the batched likelihood kernels and the
// persistent sampler: per-(theta, tile) double-float phase anchors and the
// per-bin FP32 evaluation of kappa_i = sum_k D_i(k) exp(-2 pi i phi_i(k)) over
// one slice, reduced by warp shuffles and the warp-group's shared memory.
#pragma once

#include "device_common.cuh"

namespace swig {

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Anchors of one (theta, tile) pair: A0 = frac P(f_a) (double-float sum),
// slope s = P'(f_a) df split into s_hi (x * s_hi exact for x < T) and s_lo,
// Taylor coefficients a_2..a_6 of the scaled variable x/T, and per detector
// frac(f_a tau_i).  Written as kAnchorStride floats.
__device__ inline void compute_anchor(int n_det, const TileInfo& ti, const TileBasis& tb, const EvalRecord& r,
                                      float* out) {
  dfl A = {0.0f, 0.0f}, S = {0.0f, 0.0f};
  float a[kNumPoly];
#pragma unroll
  for (int n = 0; n < kNumPoly; ++n) a[n] = 0.0f;
#pragma unroll
  for (int j = 0; j < NBASIS; ++j) {
    const dfl c = {r.c_hi[j], r.c_lo[j]};
    A = df_add(A, df_mul(c, dfl{tb.val_hi[j], tb.val_lo[j]}));
    S = df_add(S, df_mul(c, dfl{tb.slope_hi[j], tb.slope_lo[j]}));
#pragma unroll
    for (int n = 0; n < kNumPoly; ++n) a[n] = fmaf(r.c_hi[j], tb.poly[n][j], a[n]);
  }
  out[0] = df_frac(A);
  const unsigned mask = ~((1u << ti.split_bits) - 1u);
  const float s_hi = __uint_as_float(__float_as_uint(S.hi) & mask);
  out[1] = s_hi;
  out[2] = __fadd_rn(__fsub_rn(S.hi, s_hi), S.lo);
#pragma unroll
  for (int n = 0; n < kNumPoly; ++n) out[3 + n] = a[n];
  const dfl fa = {ti.fa_hi, ti.fa_lo};
#pragma unroll
  for (int i = 0; i < SWIG_MAX_DET; ++i) {
    float v = 0.0f;
    if (i < n_det) v = df_frac(df_mul(fa, dfl{r.tau_hi[i], r.tau_lo[i]}));
    out[3 + kNumPoly + i] = v;
  }
}


// Anchors of (theta, tile) held in registers by a lane; reloaded only when the
// lane crosses into the next tile (once per tile for tiles of >= 32 bins).
template <int NDET>
struct LaneAnchor {
  int end;  // first slice-local bin after the tile
  float x;  // bin offset within the tile of the lane's current bin
  float inv_T, A0, s_hi, s_lo;
  float a[kNumPoly];
  float Ad[NDET];
  // tiles and row are both indexed by row_t = t - tile_base (the tile table
  // may be a slice's copy in shared memory).
  __device__ __forceinline__ void load(const TileInfo* tiles, const float* row, int row_t, int b0, int local) {
    const TileInfo ti = tiles[row_t];
    end = ti.k0 + ti.nbins - b0;
    x = (float)(b0 + local - ti.k0);
    inv_T = ti.inv_T;
    const float* an = row + (size_t)row_t * kAnchorStride;
    A0 = an[0];
    s_hi = an[1];
    s_lo = an[2];
#pragma unroll
    for (int m = 0; m < kNumPoly; ++m) a[m] = an[3 + m];
#pragma unroll
    for (int i = 0; i < NDET; ++i) Ad[i] = an[3 + kNumPoly + i];
  }
  // Intrinsic phase (cycles) of the current bin from the tile's Taylor form.
  __device__ __forceinline__ float phase() const {
    const float u = x * inv_T;
    const float lin = x * s_hi;  // exact: s_hi carries few enough bits
    const float f1 = lin - round_nearest(lin);
    float poly = a[kNumPoly - 1];
#pragma unroll
    for (int m = kNumPoly - 2; m >= 0; --m) poly = fmaf(poly, u, a[m]);
    poly *= u * u;
    return f1 + (A0 + fmaf(x, s_lo, poly));
  }
};

// kappa_i += D_i(bin) exp(-2 pi i (p + frac(f_a tau_i) + x df tau_i)).
template <int NDET>
__device__ __forceinline__ void accumulate_bin(const LaneAnchor<NDET>& la, float p, const float* bsh,
                                               const float2* s_data, int stride, int local, float* acc_re,
                                               float* acc_im) {
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
    float ph = p + fmaf(la.x, bsh[i], la.Ad[i]);
    ph -= round_nearest(ph);
    float s, co;
    __sincosf(6.283185307179586f * ph, &s, &co);
    const float2 dv = s_data[i * stride + local];
    acc_re[i] = fmaf(dv.x, co, fmaf(dv.y, s, acc_re[i]));
    acc_im[i] = fmaf(dv.y, co, fmaf(-dv.x, s, acc_im[i]));
  }
}

// One warp evaluates the bins [b0 + lo, b0 + hi) of a slice that starts at
// bin b0, for one theta; lanes take bins lo + lane + 32 j.  s_data:
// [NDET][stride] float2 scaled D_i of the slice; s_tile: tile index of each
// slice bin; `tiles` and the anchors `row` (kAnchorStride floats per tile) are
// both indexed by (tile - tile_base).  Every lane returns the warp totals (re,
// im per detector) in out[0 .. 2 NDET).
template <int NDET>
__device__ __forceinline__ void sweep_warp_mixed(const LikeConst& L, const float2* s_data, int stride,
                                                 const int* s_tile, int b0, int lo, int hi, const TileInfo* tiles,
                                                 const float* row, int tile_base, const EvalRecord& r, int lane,
                                                 float* out) {
  float bsh[NDET];
#pragma unroll
  for (int i = 0; i < NDET; ++i) bsh[i] = (float)(L.df * r.tau[i]);
  float acc_re[NDET], acc_im[NDET];
#pragma unroll
  for (int i = 0; i < NDET; ++i) acc_re[i] = acc_im[i] = 0.0f;
  LaneAnchor<NDET> la;
  la.end = -1;
  // two bins of a tile per step (bins local and local + 32), each into its own
  // accumulators, so that a lane has two independent phase / sine / multiply-
  // add chains in flight; the two sets are added at the end
  float acc2_re[NDET], acc2_im[NDET];
#pragma unroll
  for (int i = 0; i < NDET; ++i) acc2_re[i] = acc2_im[i] = 0.0f;
  int local = lo + lane;
  while (local < hi) {
    if (local >= la.end) {
      const int t = s_tile[local];
      la.load(tiles, row, t - tile_base, b0, local);
    }
    if (local + kChunk < hi && local + kChunk < la.end) {
      const float p0 = la.phase();
      la.x += (float)kChunk;
      const float p1 = la.phase();
      la.x -= (float)kChunk;
      accumulate_bin<NDET>(la, p0, bsh, s_data, stride, local, acc_re, acc_im);
      la.x += (float)kChunk;
      accumulate_bin<NDET>(la, p1, bsh, s_data, stride, local + kChunk, acc2_re, acc2_im);
      la.x += (float)kChunk;
      local += 2 * kChunk;
    } else {
      const float p = la.phase();
      accumulate_bin<NDET>(la, p, bsh, s_data, stride, local, acc_re, acc_im);
      la.x += (float)kChunk;
      local += kChunk;
    }
  }
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
    acc_re[i] += acc2_re[i];
    acc_im[i] += acc2_im[i];
  }
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc_re[i] += __shfl_xor_sync(0xffffffffu, acc_re[i], o);
      acc_im[i] += __shfl_xor_sync(0xffffffffu, acc_im[i], o);
    }
    out[2 * i] = acc_re[i];
    out[2 * i + 1] = acc_im[i];
  }
}

// FP64 per-bin evaluation over [b0, b1) by one warp (global-memory data).
template <int NDET>
__device__ __forceinline__ void sweep_warp_fp64(const LikeConst& L, const double2* data, const double* ftab, int b0,
                                                int b1, const EvalRecord& r, int lane, double* out) {
  double acc_re[NDET], acc_im[NDET];
#pragma unroll
  for (int i = 0; i < NDET; ++i) acc_re[i] = acc_im[i] = 0.0;
  for (int bin = b0 + lane; bin < b1; bin += 32) {
    const double f = (double)(L.k_min + bin) * L.df;
    const double um = ftab[3 * (size_t)bin];      // f^-1/3
    const double up = ftab[3 * (size_t)bin + 1];  // f^1/3
    const double lf = ftab[3 * (size_t)bin + 2];  // ln f
    const double u2 = um * um, p2 = up * up;
    double P = r.c[B_ONE] + r.c[B_LOG] * lf;
    P += um * (r.c[B_M13] + um * (r.c[B_M23] + um * (r.c[B_M1] + u2 * r.c[B_M53])));
    P += up * (r.c[B_P13] + r.c[B_P13LOG] * lf) + p2 * r.c[B_P23] + p2 * p2 * up * (r.c[B_P53] + p2 * r.c[B_P73]);
#pragma unroll
    for (int i = 0; i < NDET; ++i) {
      double ph = fma(f, r.tau[i], P);
      ph -= rint(ph);
      double s, co;
      sincospi(2.0 * ph, &s, &co);
      const double2 dv = data[(size_t)i * L.n_bins + bin];
      acc_re[i] += dv.x * co + dv.y * s;
      acc_im[i] += dv.y * co - dv.x * s;
    }
  }
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc_re[i] += __shfl_xor_sync(0xffffffffu, acc_re[i], o);
      acc_im[i] += __shfl_xor_sync(0xffffffffu, acc_im[i], o);
    }
    out[2 * i] = acc_re[i];
    out[2 * i + 1] = acc_im[i];
  }
}

}  // namespace swig
