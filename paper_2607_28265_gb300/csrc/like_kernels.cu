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

#include "kernels.h"
#include "het.cuh"
#include "sweep.cuh"

namespace swig {

__global__ void k_setup(LikeConst L, const double* __restrict__ theta, int n, EvalRecord* __restrict__ rec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double th[SWIG_N_PARAMS];
  for (int j = 0; j < SWIG_N_PARAMS; ++j) th[j] = theta[(size_t)SWIG_N_PARAMS * i + j];
  if (L.dist_marg) th[6] = 1.0;   // the marginal is built from the template at 1 Mpc
  if (L.tm_n > 0) th[11] = L.tm_tref;  // templates at the fiducial's t_c, shifted node by node
  setup_record(L, th, rec + i);
}

// Per (theta, tile) anchors, one thread each (double-float on the FP32 pipe).
__global__ void k_anchor(LikeConst L, const TileInfo* __restrict__ tiles, const TileBasis* __restrict__ basis,
                         const EvalRecord* __restrict__ rec, int n, float* __restrict__ anchors) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)n * L.n_tiles;
  if (idx >= total) return;
  const int th = (int)(idx / L.n_tiles), t = (int)(idx % L.n_tiles);
  compute_anchor(L.n_det, tiles[t], basis[t], rec[th], anchors + idx * kAnchorStride);
}

// Work units are (theta, group of consecutive pieces of the slice): `groups`
// units per theta split the slice's pieces evenly, so that n * groups units
// fill the 32 warps with a small tail.  Each unit writes its own partial
// [(theta * n_slices * groups + slice * groups + unit)] (fixed reduction order).
template <int NDET>
__global__ void __launch_bounds__(kSweepThreads, 1)
    k_sweep_mixed(LikeConst L, const float2* __restrict__ data, const int* __restrict__ slice_begin,
                  const int* __restrict__ bin_tile, const TileInfo* __restrict__ tiles,
                  const float* __restrict__ anchors, const EvalRecord* __restrict__ rec, int n,
                  const int* __restrict__ piece_begin, const int* __restrict__ slice_piece, int groups,
                  float* __restrict__ partials) {
  extern __shared__ float2 s_data[];  // [NDET][slice bins], then int tile id per bin
  const int slice = blockIdx.x;
  const int b0 = slice_begin[slice], b1 = slice_begin[slice + 1];
  const int nb = b1 - b0;
  int* s_tile = reinterpret_cast<int*>(s_data + (size_t)NDET * nb);
  for (int i = 0; i < NDET; ++i)
    for (int k = threadIdx.x; k < nb; k += blockDim.x) s_data[i * nb + k] = data[(size_t)i * L.n_bins + b0 + k];
  for (int k = threadIdx.x; k < nb; k += blockDim.x) s_tile[k] = bin_tile[b0 + k];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p0 = slice_piece[slice], n_pc = slice_piece[slice + 1] - p0 - 1;
  const int g = min(groups, n_pc);
  const int units = n * groups;
  for (int u = warp; u < units; u += kSweepThreads / 32) {
    const int th = u / groups, gi = u % groups;
    float v[2 * NDET];
    if (gi < g) {
      const int pa = gi * n_pc / g, pb = (gi + 1) * n_pc / g;
      const int lo = piece_begin[p0 + pa] - b0, hi = piece_begin[p0 + pb] - b0;
      const float* row = anchors + (size_t)th * L.n_tiles * kAnchorStride;
      sweep_warp_mixed<NDET>(L, s_data, nb, s_tile, b0, lo, hi, tiles, row, 0, rec[th], lane, v);
    } else {
#pragma unroll
      for (int j = 0; j < 2 * NDET; ++j) v[j] = 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 2 * NDET; ++j)
      if (lane == j) partials[((size_t)th * L.n_slices * groups + (size_t)slice * groups + gi) * kPartialStride + j] = v[j];
  }
}

template <int NDET>
__global__ void __launch_bounds__(256)
    k_sweep_fp64(LikeConst L, const double2* __restrict__ data, const double* __restrict__ ftab,
                 const int* __restrict__ slice_begin, const EvalRecord* __restrict__ rec, int n,
                 double* __restrict__ partials) {
  const int slice = blockIdx.x;
  const int b0 = slice_begin[slice], b1 = slice_begin[slice + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int th = blockIdx.y * 8 + warp; th < n; th += gridDim.y * 8) {
    double v[2 * NDET];
    sweep_warp_fp64<NDET>(L, data, ftab, b0, b1, rec[th], lane, v);
#pragma unroll
    for (int j = 0; j < 2 * NDET; ++j)
      if (lane == j) partials[((size_t)th * L.n_slices + slice) * kPartialStride + j] = v[j];
  }
}

// Per theta: FP64 sum of the slice partials (fixed order), then the epilogue.
template <typename T>
__global__ void k_reduce(LikeConst L, const T* __restrict__ partials, int n_units, const EvalRecord* __restrict__ rec,
                         int n, double* __restrict__ out, double* __restrict__ kappa_out) {
  const int th = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (th >= n) return;
  double acc[2 * SWIG_MAX_DET];
#pragma unroll
  for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) acc[j] = 0.0;
  for (int s = lane; s < n_units; s += 32) {
    const T* p = partials + ((size_t)th * n_units + s) * kPartialStride;
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
    if (kappa_out)
      for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) kappa_out[(size_t)th * 2 * SWIG_MAX_DET + j] = acc[j];
  }
}

// ---------------------------------------------------------------------------
// Post-hoc distance of each sample of a distance-marginalised run: the
// q-quantile of p(d_L | theta, data) ~ pi(d) L(d), q from Philox-4x32-10 at
// counter (index lo, index hi, 0x64697374, 5) as a 53-bit uniform.  The
// conditional is tabulated on 1024 trapezoid cells in u = 1/d over the
// marginal's window; the quantile is read off the cumulative from the large-u
// (small-d) end and interpolated linearly inside its cell.
// ---------------------------------------------------------------------------
__global__ void k_distance_draw(LikeConst L, const EvalRecord* __restrict__ rec, const double* __restrict__ kappa,
                                int n, long long first, unsigned k0, unsigned k1, double* __restrict__ theta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const EvalRecord& r = rec[i];
  double* th = theta + (size_t)SWIG_N_PARAMS * i;
  if (!r.valid) {
    th[6] = NAN;
    return;
  }
  double zr = 0.0, zi = 0.0;
  for (int d = 0; d < L.n_det; ++d) {
    const double a = kappa[(size_t)i * 2 * SWIG_MAX_DET + 2 * d] * L.inv_scale[d];
    const double b = kappa[(size_t)i * 2 * SWIG_MAX_DET + 2 * d + 1] * L.inv_scale[d];
    zr += r.cre[d] * a - r.cim[d] * b;
    zi += r.cre[d] * b + r.cim[d] * a;
  }
  const double H = r.hh;
  const double X = L.phase_marg ? sqrt(zr * zr + zi * zi) : zr;
  double ua, ub;
  distance_window(L, X, H, &ua, &ub);
  constexpr int kCells = 1024;
  const double h = (ub - ua) / kCells;
  double M = -INFINITY;
  for (int j = 0; j <= kCells; ++j) M = fmax(M, distance_exponent(L, zr, X, H, ua + h * j));
  double total = 0.0, fprev = exp(distance_exponent(L, zr, X, H, ua) - M);
  for (int j = 1; j <= kCells; ++j) {
    const double f = exp(distance_exponent(L, zr, X, H, ua + h * j) - M);
    total += 0.5 * (f + fprev);
    fprev = f;
  }
  const long long gi = first + i;
  const uint4 w = philox4x32_10(make_uint4((unsigned)(gi & 0xFFFFFFFFll), (unsigned)(gi >> 32), 0x64697374u, 5u), k0, k1);
  const double q = ((double)(w.x >> 5) * 67108864.0 + (double)(w.y >> 6)) * (1.0 / 9007199254740992.0);
  const double target = q * total;
  double acc = 0.0, uq = ua;
  fprev = exp(distance_exponent(L, zr, X, H, ub) - M);
  for (int j = kCells - 1; j >= 0; --j) {
    const double f = exp(distance_exponent(L, zr, X, H, ua + h * j) - M);
    const double seg = 0.5 * (f + fprev);
    if (acc + seg >= target || j == 0) {
      const double frac = seg > 0.0 ? fmin(1.0, fmax(0.0, (target - acc) / seg)) : 0.5;
      uq = ua + h * (j + 1) - frac * h;
      break;
    }
    acc += seg;
    fprev = f;
  }
  th[6] = 1.0 / uq;
}

// ---------------------------------------------------------------------------
// Post-hoc t_c of time-marginalised samples (App. A): from the node log
// weights of each sample (k_het_tm's ell), the first grid node whose
// cumulative weight reaches q x total, q a 53-bit Philox uniform on the
// sample's global index (stream tag "time").  One warp per sample; the
// cumulative sums run in 32-node chunks (warp inclusive scan) in the same
// order for the total and the search, so the search always ends on a node.
// ---------------------------------------------------------------------------
__device__ inline double warp_inclusive_scan(double v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

__global__ void k_time_draw(LikeConst L, const EvalRecord* __restrict__ rec, const float* __restrict__ ell, int n,
                            long long first, unsigned k0, unsigned k1, double* __restrict__ theta) {
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double* th = theta + (size_t)SWIG_N_PARAMS * i;
  if (!rec[i].valid) {
    if (lane == 0) th[11] = NAN;
    return;
  }
  const int N = L.tm_n;
  const float* l = ell + (size_t)i * N;
  float m = -INFINITY;
  for (int j = lane; j < N; j += 32) m = fmaxf(m, l[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  double total = 0.0;
  for (int base = 0; base < N; base += 32) {
    const int j = base + lane;
    const double v = warp_inclusive_scan(j < N ? exp((double)l[j] - (double)m) : 0.0, lane);
    total += __shfl_sync(0xffffffffu, v, 31);
  }
  const long long gi = first + i;
  const uint4 w = philox4x32_10(make_uint4((unsigned)(gi & 0xFFFFFFFFll), (unsigned)(gi >> 32), 0x74696d65u, 5u), k0, k1);
  const double q = ((double)(w.x >> 5) * 67108864.0 + (double)(w.y >> 6)) * (1.0 / 9007199254740992.0);
  const double target = q * total;
  double acc = 0.0;
  int pick = N - 1;
  for (int base = 0; base < N; base += 32) {
    const int j = base + lane;
    const double v = warp_inclusive_scan(j < N ? exp((double)l[j] - (double)m) : 0.0, lane);
    const unsigned hit = __ballot_sync(0xffffffffu, j < N && acc + v >= target);
    if (hit) {
      pick = base + __ffs(hit) - 1;
      break;
    }
    acc += __shfl_sync(0xffffffffu, v, 31);
  }
  if (lane == 0) th[11] = L.tm_lo + ((double)pick + 0.5) * L.tm_dt;
}

cudaError_t launch_time_draw(const LikeConst& L, const DeviceBuffers& B, const float* ell, int n, long long first,
                             unsigned k0, unsigned k1, double* theta, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_time_draw<<<(n + 3) / 4, 128, 0, st>>>(L, B.rec, ell, n, first, k0, k1, theta);
  return cudaGetLastError();
}

cudaError_t launch_distance_draw(const LikeConst& L, const DeviceBuffers& B, const double* kappa, int n,
                                 long long first, unsigned k0, unsigned k1, double* theta, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_distance_draw<<<(n + 127) / 128, 128, 0, st>>>(L, B.rec, kappa, n, first, k0, k1, theta);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Heterodyned likelihood, one warp per theta.
// ---------------------------------------------------------------------------
template <int NDET>
__global__ void k_het(LikeConst L, HetTables H, const EvalRecord* __restrict__ rec, int n, double* __restrict__ out,
                      double* __restrict__ kappa_out, double* __restrict__ vv_out) {
  const int th = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (th >= n) return;
  const double v = het_loglike_warp<NDET>(L, H, rec[th], lane,
                                          kappa_out ? kappa_out + (size_t)th * 2 * SWIG_MAX_DET : nullptr,
                                          vv_out ? vv_out + (size_t)th * SWIG_MAX_DET : nullptr);
  if (lane == 0) out[th] = v;
}

// Time-marginalised heterodyned likelihood, one CTA per theta (the thread
// count and the chunk-to-warp assignment of the persistent sampler, so both
// give the same sums): the warps contract the bins as above, storing the edge
// products y_e in shared memory, then share the grid's 32-node chunks.
// ell (optional) receives every node's log weight, [n][tm_n].
template <int NDET>
__global__ void __launch_bounds__(kHetTmThreads, 1)
    k_het_tm(LikeConst L, HetTables H, const EvalRecord* __restrict__ rec, int n, double* __restrict__ out,
             double* __restrict__ kappa_out, double* __restrict__ vv_out, float* __restrict__ ell) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* y = reinterpret_cast<float2*>(smem);
  __shared__ float s_hh[kHetTmThreads / 32][NDET];
  __shared__ float s_tm[kHetTmThreads / 32][2];
  const int th = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  if (th >= n) return;
  const EvalRecord& r = rec[th];
  if (threadIdx.x == 0) {
    // no projection-only reuse under time marginalisation: the caches are zero
    if (kappa_out)
      for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) kappa_out[(size_t)th * 2 * SWIG_MAX_DET + j] = 0.0;
    if (vv_out)
      for (int i = 0; i < SWIG_MAX_DET; ++i) vv_out[(size_t)th * SWIG_MAX_DET + i] = 0.0;
  }
  float* ell_th = ell ? ell + (size_t)th * L.tm_n : nullptr;
  if (!r.valid) {
    if (threadIdx.x == 0) out[th] = -INFINITY;
    if (ell_th)
      for (int j = threadIdx.x; j < L.tm_n; j += blockDim.x) ell_th[j] = -INFINITY;
    return;
  }
  HetPrep<NDET> p;
  het_prepare<NDET>(L, H, r, p);
  if (L.tm_M > 0) tm_load_twiddles(L, H, smem, H.n_bins);  // read after the __syncthreads below
  float zr[NDET], zi[NDET], hh[NDET];
#pragma unroll
  for (int i = 0; i < NDET; ++i) zr[i] = zi[i] = hh[i] = 0.0f;
  const int nc = het_chunks(H.n_bins);
  for (int q = warp; q < nc; q += n_warps) het_chunk<NDET, true>(H, p, 31 * q, lane, zr, zi, hh, y);
  het_warp_reduce<NDET>(zr, zi, hh);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NDET; ++i) s_hh[warp][i] = hh[i];
  __syncthreads();
  float wm, ws;
  if (L.tm_M > 0)
    tm_pass_nufft(L, H, y, tm_nufft_grid(smem, H.n_bins), tm_nufft_tw(smem, H.n_bins, L.tm_M), warp, n_warps, lane,
                  ell_th, wm, ws);
  else
    tm_pass(L, H, y, warp, n_warps, lane, ell_th, wm, ws);
  if (lane == 0) {
    s_tm[warp][0] = wm;
    s_tm[warp][1] = ws;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double HH = 0.0;
    for (int i = 0; i < NDET; ++i) {
      double h = 0.0;
      for (int w = 0; w < n_warps; ++w) h += (double)s_hh[w][i];
      HH += h;
    }
    out[th] = tm_finish(L, s_tm, n_warps, HH);
  }
}

template <int NDET>
cudaError_t launch_het_tm(const LikeConst& L, const DeviceBuffers& B, int n, double* out, cudaStream_t st,
                          double* kappa_out, double* vv_out, float* ell) {
  const size_t bytes = het_tm_smem_bytes(B.het_nb, L.tm_M, L.tm_M > 0 ? L.tm_pieces : 0);
  cudaError_t e = cudaFuncSetAttribute(k_het_tm<NDET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_het_tm<NDET><<<n, kHetTmThreads, bytes, st>>>(L, het_tables(B), B.rec, n, out, kappa_out, vv_out, ell);
  return cudaGetLastError();
}

cudaError_t launch_loglike_het(const LikeConst& L, const DeviceBuffers& B, const double* theta, int n, double* out,
                               cudaStream_t st, double* kappa_out, double* vv_out, float* ell) {
  if (n <= 0) return cudaSuccess;
  k_setup<<<(n + 127) / 128, 128, 0, st>>>(L, theta, n, B.rec);
  if (L.tm_n > 0) {
    switch (L.n_det) {
      case 1: return launch_het_tm<1>(L, B, n, out, st, kappa_out, vv_out, ell);
      case 2: return launch_het_tm<2>(L, B, n, out, st, kappa_out, vv_out, ell);
      case 3: return launch_het_tm<3>(L, B, n, out, st, kappa_out, vv_out, ell);
      default: return launch_het_tm<4>(L, B, n, out, st, kappa_out, vv_out, ell);
    }
  }
  const HetTables H = het_tables(B);
  const unsigned grid = (unsigned)((n + 3) / 4);
  switch (L.n_det) {
    case 1: k_het<1><<<grid, 128, 0, st>>>(L, H, B.rec, n, out, kappa_out, vv_out); break;
    case 2: k_het<2><<<grid, 128, 0, st>>>(L, H, B.rec, n, out, kappa_out, vv_out); break;
    case 3: k_het<3><<<grid, 128, 0, st>>>(L, H, B.rec, n, out, kappa_out, vv_out); break;
    default: k_het<4><<<grid, 128, 0, st>>>(L, H, B.rec, n, out, kappa_out, vv_out); break;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Detector strain on the grid (FP64): h_i(f) = C_i f^-7/6 exp(-2 pi i (P(f) + f tau_i)).
// ---------------------------------------------------------------------------
__global__ void k_waveform(LikeConst L, const EvalRecord* __restrict__ rec, double2* __restrict__ out) {
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (bin >= L.n_bins || i >= L.n_det) return;
  const EvalRecord& r = rec[0];
  const double f = (double)(L.k_min + bin) * L.df;
  const double up = cbrt(f), um = 1.0 / up, lf = log(f);
  const double u2 = um * um, p2 = up * up;
  double P = r.c[B_ONE] + r.c[B_LOG] * lf;
  P += um * (r.c[B_M13] + um * (r.c[B_M23] + um * (r.c[B_M1] + u2 * r.c[B_M53])));
  P += up * (r.c[B_P13] + r.c[B_P13LOG] * lf) + p2 * r.c[B_P23] + p2 * p2 * up * (r.c[B_P53] + p2 * r.c[B_P73]);
  double ph = fma(f, r.tau[i], P);
  ph -= rint(ph);
  double s, co;
  sincospi(2.0 * ph, &s, &co);
  const double a = exp(-7.0 / 6.0 * lf);
  // C_i a (cos - i sin)
  const double re = a * (r.cre[i] * co + r.cim[i] * s), im = a * (r.cim[i] * co - r.cre[i] * s);
  out[(size_t)i * L.n_bins + bin] = make_double2(re, im);
}

cudaError_t launch_waveform(const LikeConst& L, const double* theta_dev, EvalRecord* rec_dev, double2* out,
                            cudaStream_t st) {
  k_setup<<<1, 32, 0, st>>>(L, theta_dev, 1, rec_dev);
  dim3 grid((L.n_bins + 255) / 256, L.n_det);
  k_waveform<<<grid, 256, 0, st>>>(L, rec_dev, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prior transform (Table I inverse CDFs).
// ---------------------------------------------------------------------------
__global__ void k_prior_transform(const PriorSlot* __restrict__ slots, int n_sampled, const double* __restrict__ u,
                                  int n, double* __restrict__ theta, SkyFrame sky) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  prior_map(slots, u + (size_t)i * n_sampled, theta + (size_t)i * SWIG_N_PARAMS, &sky);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_loglike_mixed(const LikeConst& L, const DeviceBuffers& B, const double* theta, int n,
                                 double* out, cudaStream_t st, double* kappa_out) {
  if (n <= 0) return cudaSuccess;
  k_setup<<<(n + 127) / 128, 128, 0, st>>>(L, theta, n, B.rec);
  const long long items = (long long)n * L.n_tiles;
  k_anchor<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(L, B.tiles, B.basis, B.rec, n, B.anchors);
  const size_t smem = sweep_smem_bytes(L.n_det, B.max_slice_bins);
  // units per theta: the smallest g whose tail over 32 warps is below ~10%
  int groups = 1;
  for (int gg = 1; gg <= 4; ++gg) {
    groups = gg;
    const int units = n * gg, waves = (units + 31) / 32;
    if ((double)units / (32.0 * waves) >= 0.9) break;
  }
  switch (L.n_det) {
    case 1: k_sweep_mixed<1><<<L.n_slices, kSweepThreads, smem, st>>>(L, B.data32, B.slice_begin, B.bin_tile, B.tiles, B.anchors, B.rec, n, B.piece_begin, B.slice_piece, groups, B.partials32); break;
    case 2: k_sweep_mixed<2><<<L.n_slices, kSweepThreads, smem, st>>>(L, B.data32, B.slice_begin, B.bin_tile, B.tiles, B.anchors, B.rec, n, B.piece_begin, B.slice_piece, groups, B.partials32); break;
    case 3: k_sweep_mixed<3><<<L.n_slices, kSweepThreads, smem, st>>>(L, B.data32, B.slice_begin, B.bin_tile, B.tiles, B.anchors, B.rec, n, B.piece_begin, B.slice_piece, groups, B.partials32); break;
    default: k_sweep_mixed<4><<<L.n_slices, kSweepThreads, smem, st>>>(L, B.data32, B.slice_begin, B.bin_tile, B.tiles, B.anchors, B.rec, n, B.piece_begin, B.slice_piece, groups, B.partials32); break;
  }
  k_reduce<float><<<(n + 3) / 4, 128, 0, st>>>(L, B.partials32, L.n_slices * groups, B.rec, n, out, kappa_out);
  return cudaGetLastError();
}

cudaError_t launch_loglike_fp64(const LikeConst& L, const DeviceBuffers& B, const double* theta, int n,
                                double* out, cudaStream_t st, double* kappa_out) {
  if (n <= 0) return cudaSuccess;
  k_setup<<<(n + 127) / 128, 128, 0, st>>>(L, theta, n, B.rec);
  const int gy = (n + 7) / 8 < 64 ? (n + 7) / 8 : 64;
  dim3 grid(L.n_slices, gy);
  switch (L.n_det) {
    case 1: k_sweep_fp64<1><<<grid, 256, 0, st>>>(L, B.data64, B.ftab, B.slice_begin, B.rec, n, B.partials64); break;
    case 2: k_sweep_fp64<2><<<grid, 256, 0, st>>>(L, B.data64, B.ftab, B.slice_begin, B.rec, n, B.partials64); break;
    case 3: k_sweep_fp64<3><<<grid, 256, 0, st>>>(L, B.data64, B.ftab, B.slice_begin, B.rec, n, B.partials64); break;
    default: k_sweep_fp64<4><<<grid, 256, 0, st>>>(L, B.data64, B.ftab, B.slice_begin, B.rec, n, B.partials64); break;
  }
  k_reduce<double><<<(n + 3) / 4, 128, 0, st>>>(L, B.partials64, L.n_slices, B.rec, n, out, kappa_out);
  return cudaGetLastError();
}

cudaError_t launch_prior_transform(const PriorSlot* slots, int n_sampled, const double* u, int n, double* theta,
                                   cudaStream_t st, SkyFrame sky) {
  if (n <= 0) return cudaSuccess;
  k_prior_transform<<<(n + 127) / 128, 128, 0, st>>>(slots, n_sampled, u, n, theta, sky);
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
