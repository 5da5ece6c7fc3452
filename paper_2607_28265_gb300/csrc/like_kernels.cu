// Batched matched-filter log-likelihood kernels (Eq. 2 of the paper) on the
// full frequency grid, in two precisions:
//
//  * MIXED: per-bin work in FP32.  The TaylorF2 phase is anchored per tile in
//    double-float (FP32 pairs): within a tile of T bins the phase in cycles is
//    P(f_a + x df) = A0 + frac(x s_hi) + x s_lo + sum_{n=2..6} a_n (x/T)^n with
//    A0 = frac P(f_a), s = P'(f_a) df split so that x s_hi is exact, and the
//    Taylor coefficients a_n from the tile's basis table.  Each detector adds
//    frac(f_a tau_i) + x df tau_i.  The complex exponential uses the SFU
//    (__sincosf on the reduced argument), the per-bin products are
//    accumulated in FP32 per thread and combined by a pairwise tree (warp
//    shuffles, shared memory, then FP64 across slices).
//  * FP64: every per-bin quantity in FP64 with sincospi, as the reference
//    precision of the small single-detector configuration.
//
// The grid is cut into `n_slices` contiguous ranges of whole 32-bin chunks,
// one CTA per slice; the slice's data D_i(f) = 4 df conj(d_i) f^-7/6 / S_i is
// staged once into shared memory and reused for every theta of the batch.
// Inside a CTA each warp-group (4 warps) evaluates one theta at a time over the
// slice and writes one partial sum per (theta, slice).
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace swig {

__global__ void k_setup(LikeConst L, const double* __restrict__ theta, int n, EvalRecord* __restrict__ rec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) setup_record(L, theta + (size_t)SWIG_N_PARAMS * i, rec + i);
}

// Per (theta, tile) anchors, one thread each (double-float on the FP32 pipe).
__device__ inline void compute_anchor(const LikeConst& L, const TileInfo& ti, const TileBasis& tb,
                                      const EvalRecord& r, float* out) {
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
  // slope split: clear `split_bits` low mantissa bits so x * s_hi is exact for x < T
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
    if (i < L.n_det) v = df_frac(df_mul(fa, dfl{r.tau_hi[i], r.tau_lo[i]}));
    out[3 + kNumPoly + i] = v;
  }
}

__global__ void k_anchor(LikeConst L, const TileInfo* __restrict__ tiles, const TileBasis* __restrict__ basis,
                         const EvalRecord* __restrict__ rec, int n, float* __restrict__ anchors) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)n * L.n_tiles;
  if (idx >= total) return;
  const int th = (int)(idx / L.n_tiles), t = (int)(idx % L.n_tiles);
  compute_anchor(L, tiles[t], basis[t], rec[th], anchors + idx * kAnchorStride);
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Anchors of (theta, tile) held in registers by each lane; reloaded only when
// the lane's tile changes (once per tile for tiles of >= 32 bins).
template <int NDET>
struct LaneAnchor {
  int tile;
  int k0;
  float inv_T, A0, s_hi, s_lo;
  float a[kNumPoly];
  float Ad[NDET];
  __device__ __forceinline__ void load(const TileInfo* tiles, const float* anchors, size_t th_off, int t) {
    tile = t;
    k0 = tiles[t].k0;
    inv_T = tiles[t].inv_T;
    const float* an = anchors + (th_off + t) * kAnchorStride;
    A0 = an[0];
    s_hi = an[1];
    s_lo = an[2];
#pragma unroll
    for (int m = 0; m < kNumPoly; ++m) a[m] = an[3 + m];
#pragma unroll
    for (int i = 0; i < NDET; ++i) Ad[i] = an[3 + kNumPoly + i];
  }
};

template <int NDET>
__global__ void __launch_bounds__(kSweepThreads, 1)
    k_sweep_mixed(LikeConst L, const float2* __restrict__ data, const int* __restrict__ slice_begin,
                  const int* __restrict__ bin_tile, const TileInfo* __restrict__ tiles,
                  const float* __restrict__ anchors, const EvalRecord* __restrict__ rec, int n,
                  float* __restrict__ partials) {
  extern __shared__ float2 s_data[];  // [NDET][slice bins], then int tile id per bin
  __shared__ float s_red[kWarpGroups][4][2 * NDET];
  const int slice = blockIdx.x;
  const int b0 = slice_begin[slice], b1 = slice_begin[slice + 1];
  const int nb = b1 - b0;
  int* s_tile = reinterpret_cast<int*>(s_data + (size_t)NDET * nb);
  for (int i = 0; i < NDET; ++i)
    for (int k = threadIdx.x; k < nb; k += blockDim.x) s_data[i * nb + k] = data[(size_t)i * L.n_bins + b0 + k];
  for (int k = threadIdx.x; k < nb; k += blockDim.x) s_tile[k] = bin_tile[b0 + k];
  __syncthreads();

  const int wg = threadIdx.x >> 7, wl = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;
  // each warp of a group owns a contiguous run of 32-bin chunks of the slice
  const int n_ch = (nb + kChunk - 1) / kChunk;
  const int per_warp = (n_ch + 3) / 4;
  const int cw0 = wl * per_warp, cw1 = min(cw0 + per_warp, n_ch);
  const float twopi = 6.283185307179586f;
  for (int th = wg; th < n; th += kWarpGroups) {
    const EvalRecord& r = rec[th];
    const size_t th_off = (size_t)th * L.n_tiles;
    float bsh[NDET];
#pragma unroll
    for (int i = 0; i < NDET; ++i) bsh[i] = (float)(L.df * r.tau[i]);
    float acc_re[NDET], acc_im[NDET];
#pragma unroll
    for (int i = 0; i < NDET; ++i) acc_re[i] = acc_im[i] = 0.0f;
    LaneAnchor<NDET> la;
    la.tile = -1;
    for (int cc = cw0; cc < cw1; ++cc) {
      const int local = cc * kChunk + lane;
      if (local < nb) {
        const int t = s_tile[local];
        if (t != la.tile) la.load(tiles, anchors, th_off, t);
        const float x = (float)(b0 + local - la.k0);
        const float u = x * la.inv_T;
        const float lin = x * la.s_hi;  // exact: s_hi has few enough bits
        const float f1 = lin - rintf(lin);
        float poly = la.a[kNumPoly - 1];
#pragma unroll
        for (int m = kNumPoly - 2; m >= 0; --m) poly = fmaf(poly, u, la.a[m]);
        poly *= u * u;
        const float p = f1 + (la.A0 + fmaf(x, la.s_lo, poly));
#pragma unroll
        for (int i = 0; i < NDET; ++i) {
          float ph = p + fmaf(x, bsh[i], la.Ad[i]);
          ph -= rintf(ph);
          float s, co;
          __sincosf(twopi * ph, &s, &co);
          const float2 dv = s_data[i * nb + local];
          acc_re[i] = fmaf(dv.x, co, fmaf(dv.y, s, acc_re[i]));
          acc_im[i] = fmaf(dv.y, co, fmaf(-dv.x, s, acc_im[i]));
        }
      }
    }
    // pairwise tree: warp shuffles, then the 4 warps of the group
#pragma unroll
    for (int i = 0; i < NDET; ++i) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc_re[i] += __shfl_xor_sync(0xffffffffu, acc_re[i], o);
        acc_im[i] += __shfl_xor_sync(0xffffffffu, acc_im[i], o);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < NDET; ++i) {
        s_red[wg][wl][2 * i] = acc_re[i];
        s_red[wg][wl][2 * i + 1] = acc_im[i];
      }
    }
    named_barrier(1 + wg, 128);
    if (wl == 0 && lane < 2 * NDET) {
      const float v = (s_red[wg][0][lane] + s_red[wg][1][lane]) + (s_red[wg][2][lane] + s_red[wg][3][lane]);
      partials[((size_t)th * L.n_slices + slice) * kPartialStride + lane] = v;
    }
    named_barrier(1 + wg, 128);
  }
}

template <int NDET>
__global__ void __launch_bounds__(256)
    k_sweep_fp64(LikeConst L, const double2* __restrict__ data, const double* __restrict__ ftab,
                 const int* __restrict__ slice_begin, const EvalRecord* __restrict__ rec, int n,
                 double* __restrict__ partials) {
  __shared__ double s_red[2][4][2 * NDET];
  const int slice = blockIdx.x;
  const int b0 = slice_begin[slice], b1 = slice_begin[slice + 1];
  const int wg = threadIdx.x >> 7, wl = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;
  const int tid = threadIdx.x & 127;
  for (int th = blockIdx.y * 2 + wg; th < n; th += gridDim.y * 2) {
    const EvalRecord& r = rec[th];
    double acc_re[NDET], acc_im[NDET];
#pragma unroll
    for (int i = 0; i < NDET; ++i) acc_re[i] = acc_im[i] = 0.0;
    for (int bin = b0 + tid; bin < b1; bin += 128) {
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
    }
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < NDET; ++i) {
        s_red[wg][wl][2 * i] = acc_re[i];
        s_red[wg][wl][2 * i + 1] = acc_im[i];
      }
    }
    named_barrier(1 + wg, 128);
    if (wl == 0 && lane < 2 * NDET) {
      const double v = (s_red[wg][0][lane] + s_red[wg][1][lane]) + (s_red[wg][2][lane] + s_red[wg][3][lane]);
      partials[((size_t)th * L.n_slices + slice) * kPartialStride + lane] = v;
    }
    named_barrier(1 + wg, 128);
  }
}

// Per theta: FP64 sum of the slice partials (fixed order), then the epilogue.
template <typename T>
__global__ void k_reduce(LikeConst L, const T* __restrict__ partials, const EvalRecord* __restrict__ rec, int n,
                         double* __restrict__ out) {
  const int th = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (th >= n) return;
  double acc[2 * SWIG_MAX_DET];
#pragma unroll
  for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) acc[j] = 0.0;
  for (int s = lane; s < L.n_slices; s += 32) {
    const T* p = partials + ((size_t)th * L.n_slices + s) * kPartialStride;
#pragma unroll
    for (int j = 0; j < 2 * SWIG_MAX_DET; ++j)
      if (j < 2 * L.n_det) acc[j] += (double)p[j];
  }
#pragma unroll
  for (int j = 0; j < 2 * SWIG_MAX_DET; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  if (lane == 0) {
    double kre[SWIG_MAX_DET], kim[SWIG_MAX_DET];
    for (int i = 0; i < SWIG_MAX_DET; ++i) {
      kre[i] = acc[2 * i];
      kim[i] = acc[2 * i + 1];
    }
    out[th] = loglike_epilogue(L, rec[th], kre, kim);
  }
}

// ---------------------------------------------------------------------------
// Prior transform (Table I inverse CDFs).
// ---------------------------------------------------------------------------
__global__ void k_prior_transform(const PriorSlot* __restrict__ slots, int n_sampled, const double* __restrict__ u,
                                  int n, double* __restrict__ theta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  prior_map(slots, u + (size_t)i * n_sampled, theta + (size_t)i * SWIG_N_PARAMS);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_loglike_mixed(const LikeConst& L, const DeviceBuffers& B, const double* theta, int n,
                                 double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_setup<<<(n + 127) / 128, 128, 0, st>>>(L, theta, n, B.rec);
  const long long items = (long long)n * L.n_tiles;
  k_anchor<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(L, B.tiles, B.basis, B.rec, n, B.anchors);
  const size_t smem = sweep_smem_bytes(L.n_det, B.max_slice_bins);
  switch (L.n_det) {
    case 1: k_sweep_mixed<1><<<L.n_slices, kSweepThreads, smem, st>>>(L, B.data32, B.slice_begin, B.bin_tile, B.tiles, B.anchors, B.rec, n, B.partials32); break;
    case 2: k_sweep_mixed<2><<<L.n_slices, kSweepThreads, smem, st>>>(L, B.data32, B.slice_begin, B.bin_tile, B.tiles, B.anchors, B.rec, n, B.partials32); break;
    case 3: k_sweep_mixed<3><<<L.n_slices, kSweepThreads, smem, st>>>(L, B.data32, B.slice_begin, B.bin_tile, B.tiles, B.anchors, B.rec, n, B.partials32); break;
    default: k_sweep_mixed<4><<<L.n_slices, kSweepThreads, smem, st>>>(L, B.data32, B.slice_begin, B.bin_tile, B.tiles, B.anchors, B.rec, n, B.partials32); break;
  }
  k_reduce<float><<<(n + 3) / 4, 128, 0, st>>>(L, B.partials32, B.rec, n, out);
  return cudaGetLastError();
}

cudaError_t launch_loglike_fp64(const LikeConst& L, const DeviceBuffers& B, const double* theta, int n,
                                double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_setup<<<(n + 127) / 128, 128, 0, st>>>(L, theta, n, B.rec);
  const int gy = (n + 1) / 2 < 64 ? (n + 1) / 2 : 64;
  dim3 grid(L.n_slices, gy);
  switch (L.n_det) {
    case 1: k_sweep_fp64<1><<<grid, 256, 0, st>>>(L, B.data64, B.ftab, B.slice_begin, B.rec, n, B.partials64); break;
    case 2: k_sweep_fp64<2><<<grid, 256, 0, st>>>(L, B.data64, B.ftab, B.slice_begin, B.rec, n, B.partials64); break;
    case 3: k_sweep_fp64<3><<<grid, 256, 0, st>>>(L, B.data64, B.ftab, B.slice_begin, B.rec, n, B.partials64); break;
    default: k_sweep_fp64<4><<<grid, 256, 0, st>>>(L, B.data64, B.ftab, B.slice_begin, B.rec, n, B.partials64); break;
  }
  k_reduce<double><<<(n + 3) / 4, 128, 0, st>>>(L, B.partials64, B.rec, n, out);
  return cudaGetLastError();
}

cudaError_t launch_prior_transform(const PriorSlot* slots, int n_sampled, const double* u, int n, double* theta,
                                   cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_prior_transform<<<(n + 127) / 128, 128, 0, st>>>(slots, n_sampled, u, n, theta);
  return cudaGetLastError();
}

cudaError_t set_sweep_smem_limit(size_t bytes) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_sweep_mixed<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes))) return e;
  if ((e = cudaFuncSetAttribute(k_sweep_mixed<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes))) return e;
  if ((e = cudaFuncSetAttribute(k_sweep_mixed<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes))) return e;
  return cudaFuncSetAttribute(k_sweep_mixed<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace swig
