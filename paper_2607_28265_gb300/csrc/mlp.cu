// Learned slice proposal on the device: initialisation, training targets,
// BF16 tensor-core matrix products (FP32 accumulation), loss, Adam, and a
// captured CUDA graph for the training step.  See mlp.h for the model.
//
// Every kernel is deterministic (fixed summation orders, split-K partials
// summed in split order); the same inputs give bit-identical parameters.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include "device_common.cuh"
#include "mlp.h"

namespace swig {

namespace {

constexpr int kGemmTile = 64;
constexpr int kGemmThreads = 128;
constexpr int kTargetWarps = 4;
constexpr int kMaxNbr = 2 * kMlpIn;
constexpr int kPowerIters = 600;

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// ---------------------------------------------------------------------------
// Initial weights: W[i][j] = Box-Muller(Philox(j, i, layer, 9)) / sqrt(fan_in)
// ---------------------------------------------------------------------------
__global__ void k_mlp_init(float* params, unsigned k0, unsigned k1) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  int layer, fan_in, cols, base;
  if (p < kMlpOffB1) {
    layer = 0, fan_in = kMlpIn, cols = kMlpH, base = kMlpOffW1;
  } else if (p < kMlpOffW2) {
    params[p] = 0.0f;
    return;
  } else if (p < kMlpOffB2) {
    layer = 2, fan_in = kMlpH, cols = kMlpH, base = kMlpOffW2;
  } else if (p < kMlpOffW3) {
    params[p] = 0.0f;
    return;
  } else if (p < kMlpOffB3) {
    layer = 4, fan_in = kMlpH, cols = kMlpOut, base = kMlpOffW3;
  } else {
    params[p] = 0.0f;
    return;
  }
  const int q = p - base, i = q / cols, j = q % cols;
  const uint4 r = philox4x32_10(make_uint4((unsigned)j, (unsigned)i, (unsigned)layer, 9u), k0, k1);
  const double u1 = ((double)(r.x >> 8) + 1.0) * (1.0 / 16777216.0);
  const double u2 = (double)(r.y >> 8) * (1.0 / 16777216.0);
  params[p] = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2) / sqrt((double)fan_in));
}

// BF16 copies of the weights in the padded layouts of the matrix products.
__device__ __forceinline__ void write_bf16_weight(int p, float w, __nv_bfloat16* w1b, __nv_bfloat16* w2b,
                                                  __nv_bfloat16* w3b) {
  if (p < kMlpOffB1) {
    w1b[p - kMlpOffW1] = __float2bfloat16_rn(w);  // [13][256] inside [16][256]
  } else if (p >= kMlpOffW2 && p < kMlpOffB2) {
    w2b[p - kMlpOffW2] = __float2bfloat16_rn(w);
  } else if (p >= kMlpOffW3 && p < kMlpOffB3) {
    const int q = p - kMlpOffW3;
    w3b[(q / kMlpOut) * kMlpOutPad + q % kMlpOut] = __float2bfloat16_rn(w);
  }
}

__global__ void k_mlp_bf16_weights(const float* params, __nv_bfloat16* w1b, __nv_bfloat16* w2b, __nv_bfloat16* w3b) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) write_bf16_weight(p, params[p], w1b, w2b, w3b);
}

// ---------------------------------------------------------------------------
// Live-set statistics, network inputs and local-PCA targets
// ---------------------------------------------------------------------------
// mean and population standard deviation (floored at 1e-12) per dimension;
// one warp per dimension, fixed-order lane sums and shuffle tree
__global__ void k_live_stats(const double* u, int n, int d, double* stats) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w >= d) return;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += u[(size_t)i * d + w];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const double mu = s / (double)n;
  double v = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double t = u[(size_t)i * d + w] - mu;
    v += t * t;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) {
    stats[w] = mu;
    stats[kMlpIn + w] = fmax(sqrt(v / (double)n), 1e-12);
  }
}

// standardised coordinates (FP64, n x d) and the BF16 network inputs (n x 16)
__global__ void k_standardise(const double* u, int n, int d, const double* stats, double* xs, __nv_bfloat16* xb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * kMlpInPad) return;
  const int i = e / kMlpInPad, j = e % kMlpInPad;
  if (j < d) {
    const double x = (u[(size_t)i * d + j] - stats[j]) / stats[kMlpIn + j];
    xs[(size_t)i * d + j] = x;
    xb[e] = __float2bfloat16_rn((float)x);
  } else {
    xb[e] = __float2bfloat16_rn(0.0f);
  }
}

__global__ void k_inputs_f32(const float* x, int n, __nv_bfloat16* xb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * kMlpInPad) return;
  const int i = e / kMlpInPad, j = e % kMlpInPad;
  xb[e] = __float2bfloat16_rn(j < kMlpIn ? x[(size_t)i * kMlpIn + j] : 0.0f);
}

// One warp per live point: the k nearest other points in standardised
// coordinates (ties by index), their covariance in unit-cube coordinates, log
// standard deviations, and the leading eigenvector of the correlation matrix
// by power iteration (sign: largest-magnitude entry positive).
__global__ void __launch_bounds__(32 * kTargetWarps) k_local_pca(const double* u, const double* xs, int n, int d, int k,
                                                               float* tdir, float* tls, int* nbr) {
  __shared__ int s_nb[kTargetWarps][kMaxNbr];
  __shared__ double s_c[kTargetWarps][kMlpIn * kMlpIn];
  __shared__ double s_v[kTargetWarps][kMlpIn];
  __shared__ double s_mean[kTargetWarps][kMlpIn];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kTargetWarps + w;
  if (i >= n) return;
  double xi[kMlpIn];
  for (int q = 0; q < d; ++q) xi[q] = xs[(size_t)i * d + q];
  double last_d = -1.0;
  int last_j = -1;
  for (int r = 0; r < k; ++r) {
    double bd = INFINITY;
    int bj = INT_MAX;
    for (int j = lane; j < n; j += 32) {
      if (j == i) continue;
      double dd = 0.0;
      for (int q = 0; q < d; ++q) {
        const double t = xs[(size_t)j * d + q] - xi[q];
        dd += t * t;
      }
      const bool after = dd > last_d || (dd == last_d && j > last_j);
      const bool better = dd < bd || (dd == bd && j < bj);
      if (after && better) {
        bd = dd;
        bj = j;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double od = __shfl_xor_sync(0xffffffffu, bd, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (od < bd || (od == bd && oj < bj)) {
        bd = od;
        bj = oj;
      }
    }
    last_d = bd;
    last_j = bj;
    if (lane == 0) s_nb[w][r] = bj;
  }
  __syncwarp();
  // covariance of the neighbours (1/k normalisation)
  if (lane < d) {
    double s = 0.0;
    for (int r = 0; r < k; ++r) s += u[(size_t)s_nb[w][r] * d + lane];
    s_mean[w][lane] = s / (double)k;
  }
  __syncwarp();
  for (int e = lane; e < d * d; e += 32) {
    const int a = e / d, b = e % d;
    double s = 0.0;
    for (int r = 0; r < k; ++r) {
      const size_t row = (size_t)s_nb[w][r] * d;
      s += (u[row + a] - s_mean[w][a]) * (u[row + b] - s_mean[w][b]);
    }
    s_c[w][e] = s / (double)k;
  }
  __syncwarp();
  double sig = 1.0;
  if (lane < d) sig = fmax(sqrt(s_c[w][lane * d + lane]), 1e-12);
  // row of the correlation matrix R_ab = C_ab / (sig_a sig_b) in registers
  double ra[kMlpIn];
  if (lane < d) {
    for (int b = 0; b < d; ++b) {
      const double sb = fmax(sqrt(s_c[w][b * d + b]), 1e-12);
      ra[b] = s_c[w][lane * d + b] / (sig * sb);
    }
    s_v[w][lane] = 1.0 / sqrt((double)d);
  }
  __syncwarp();
  for (int it = 0; it < kPowerIters; ++it) {
    double y = 0.0;
    if (lane < d)
      for (int b = 0; b < d; ++b) y += ra[b] * s_v[w][b];
    double nn = lane < d ? y * y : 0.0;
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    __syncwarp();
    if (lane < d) s_v[w][lane] = nn > 0.0 ? y / sqrt(nn) : s_v[w][lane];
    __syncwarp();
  }
  // sign: the largest-magnitude entry (first on ties) positive
  double best = -1.0;
  int arg = 0;
  for (int b = 0; b < d; ++b) {
    const double a = fabs(s_v[w][b]);
    if (a > best) {
      best = a;
      arg = b;
    }
  }
  const double sgn = s_v[w][arg] < 0.0 ? -1.0 : 1.0;
  if (lane < kMlpIn) {
    tdir[(size_t)i * kMlpIn + lane] = lane < d ? (float)(sgn * s_v[w][lane]) : 0.0f;
    tls[(size_t)i * kMlpIn + lane] = lane < d ? (float)log(sig) : 0.0f;
  }
  if (lane < k && nbr) nbr[(size_t)i * kMaxNbr + lane] = s_nb[w][lane];
}

// ---------------------------------------------------------------------------
// C[z] = sum_{k in split z} A(i, k) B(k, j): BF16 operands through strides,
// FP32 accumulation with mma.sync m16n8k16; 64 x 64 tile per 4 warps.
// ---------------------------------------------------------------------------
struct GemmDesc {
  const __nv_bfloat16* A;
  long long a_si, a_sk;
  const __nv_bfloat16* B;
  long long b_sk, b_sj;
  int M, N, K, k_split;
  float* part;  // [splits][M][N]
};

__device__ __forceinline__ void mma_bf16_16816(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(kGemmThreads) k_gemm_bf16(GemmDesc g) {
  __shared__ __align__(16) __nv_bfloat16 As[kGemmTile][24];  // [row][k]
  __shared__ __align__(16) __nv_bfloat16 Bs[kGemmTile][24];  // [col][k]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kGemmTile, n0 = blockIdx.x * kGemmTile, z = blockIdx.z;
  const int kbeg = z * g.k_split, kend = min(g.K, kbeg + g.k_split);
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int e = tid; e < kGemmTile * 16; e += kGemmThreads) {
      const int r = e >> 4, kk = e & 15, i = m0 + r, kx = k0 + kk;
      As[r][kk] = (i < g.M && kx < kend) ? g.A[(long long)i * g.a_si + (long long)kx * g.a_sk] : zero;
      const int j = n0 + r;
      Bs[r][kk] = (j < g.N && kx < kend) ? g.B[(long long)kx * g.b_sk + (long long)j * g.b_sj] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
      const int r = wm + mi * 16;
      unsigned a[4];
      a[0] = *reinterpret_cast<const unsigned*>(&As[r + gid][2 * tig]);
      a[1] = *reinterpret_cast<const unsigned*>(&As[r + gid + 8][2 * tig]);
      a[2] = *reinterpret_cast<const unsigned*>(&As[r + gid][2 * tig + 8]);
      a[3] = *reinterpret_cast<const unsigned*>(&As[r + gid + 8][2 * tig + 8]);
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c = wn + ni * 8;
        unsigned b[2];
        b[0] = *reinterpret_cast<const unsigned*>(&Bs[c + gid][2 * tig]);
        b[1] = *reinterpret_cast<const unsigned*>(&Bs[c + gid][2 * tig + 8]);
        mma_bf16_16816(acc[mi][ni], a, b);
      }
    }
    __syncthreads();
  }
  float* out = g.part + (size_t)z * g.M * g.N;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = m0 + wm + mi * 16 + gid + 8 * h;
        const int col = n0 + wn + ni * 8 + 2 * tig;
        if (row < g.M) {
          if (col < g.N) out[(size_t)row * g.N + col] = acc[mi][ni][2 * h];
          if (col + 1 < g.N) out[(size_t)row * g.N + col + 1] = acc[mi][ni][2 * h + 1];
        }
      }
}

enum EpiMode { EPI_PLAIN = 0, EPI_HIDDEN = 1, EPI_BACK = 2 };

struct EpiDesc {
  const float* part;
  int splits, M, N, mode;
  const float* bias;  // [N] or null
  const float* zin;   // EPI_BACK: pre-activation, row stride ld_z
  int ld_z;
  float* out32;  // row stride ld_out
  int ld_out;
  __nv_bfloat16* outb;  // row stride ld_outb (EPI_HIDDEN: bf16(silu); EPI_BACK: bf16(value))
  int ld_outb;
};

__global__ void k_gemm_epi(EpiDesc e) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)e.M * e.N) return;
  const int i = (int)(idx / e.N), j = (int)(idx % e.N);
  float v = 0.0f;
  for (int z = 0; z < e.splits; ++z) v += e.part[((size_t)z * e.M + i) * e.N + j];
  if (e.mode == EPI_PLAIN) {
    if (e.bias) v += e.bias[j];
    e.out32[(size_t)i * e.ld_out + j] = v;
  } else if (e.mode == EPI_HIDDEN) {
    v += e.bias[j];
    e.out32[(size_t)i * e.ld_out + j] = v;
    e.outb[(size_t)i * e.ld_outb + j] = __float2bfloat16_rn(silu_f(v));
  } else {
    v *= dsilu_f(e.zin[(size_t)i * e.ld_z + j]);
    e.out32[(size_t)i * e.ld_out + j] = v;
    e.outb[(size_t)i * e.ld_outb + j] = __float2bfloat16_rn(v);
  }
}

// ---------------------------------------------------------------------------
// Loss, bias gradients, Adam
// ---------------------------------------------------------------------------
__global__ void k_mlp_loss(const float* out, const float* tdir, const float* tls, int n, int d, float* dout,
                           __nv_bfloat16* doutb, double* row_loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* o = out + (size_t)i * kMlpOutPad;
  const float* t = tdir + (size_t)i * kMlpIn;
  const float* ls = tls + (size_t)i * kMlpIn;
  float nrm2 = 0.0f;
  for (int j = 0; j < d; ++j) nrm2 += o[j] * o[j];
  const float nrm = sqrtf(nrm2 + 1e-12f);
  float c = 0.0f;
  for (int j = 0; j < d; ++j) c += (o[j] / nrm) * t[j];
  double l = 1.0 - (double)c * (double)c;
  const float inv_n = 1.0f / (float)n;
  float* g = dout + (size_t)i * kMlpOutPad;
  __nv_bfloat16* gb = doutb + (size_t)i * kMlpOutPad;
  for (int j = 0; j < kMlpOutPad; ++j) {
    float v = 0.0f;
    if (j < d) {
      v = -2.0f * c * (t[j] - c * (o[j] / nrm)) / nrm * inv_n;
    } else if (j >= kMlpIn && j < kMlpIn + d) {
      const float df = o[j] - ls[j - kMlpIn];
      l += (double)df * (double)df;
      v = 2.0f * df * inv_n;
    }
    g[j] = v;
    gb[j] = __float2bfloat16_rn(v);
  }
  row_loss[i] = l;
}

// deterministic mean of row_loss (one block, fixed tree)
__global__ void k_mean(const double* v, int n, double* out) {
  __shared__ double s[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += v[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0] / (double)n;
}

// column sums over rows (FP64, row order) into FP32 gradients
__global__ void k_col_sum(const float* src, int n, int ld, int ncols, float* dst) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += src[(size_t)i * ld + j];
  dst[j] = (float)s;
}

__global__ void k_adam(float* params, const float* grad, float* m, float* v, const int* step, float lr,
                       __nv_bfloat16* w1b, __nv_bfloat16* w2b, __nv_bfloat16* w3b) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int t = *step + 1;
  const float g = grad[p];
  const float mm = b1 * m[p] + (1.0f - b1) * g;
  const float vv = b2 * v[p] + (1.0f - b2) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / (1.0f - powf(b1, (float)t));
  const float vh = vv / (1.0f - powf(b2, (float)t));
  const float w = params[p] - lr * mh / (sqrtf(vh) + eps);
  params[p] = w;
  write_bf16_weight(p, w, w1b, w2b, w3b);
}

__global__ void k_step_inc(int* step) { *step += 1; }

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t dalloc(T*& p, size_t n) {
  return cudaMalloc(&p, sizeof(T) * (n ? n : 1));
}

cudaError_t gemm(Mlp& M, const __nv_bfloat16* A, long long a_si, long long a_sk, const __nv_bfloat16* B,
                 long long b_sk, long long b_sj, int m, int n, int k, EpiDesc epi, cudaStream_t st, long long* L) {
  int splits = 1;
  if (k >= 512 && (long long)m * n <= (long long)kMlpH * kMlpH) splits = std::min(kMlpMaxSplit, k / 256);
  int ks = (k + splits - 1) / splits;
  ks = (ks + 15) / 16 * 16;
  splits = (k + ks - 1) / ks;
  GemmDesc g{A, a_si, a_sk, B, b_sk, b_sj, m, n, k, ks, M.part};
  dim3 grid((n + kGemmTile - 1) / kGemmTile, (m + kGemmTile - 1) / kGemmTile, splits);
  k_gemm_bf16<<<grid, kGemmThreads, 0, st>>>(g);
  epi.part = M.part;
  epi.splits = splits;
  epi.M = m;
  epi.N = n;
  const long long tot = (long long)m * n;
  k_gemm_epi<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(epi);
  if (L) *L += 2;
  return cudaGetLastError();
}

EpiDesc epi_plain(const float* bias, float* out, int ld) {
  EpiDesc e{};
  e.mode = EPI_PLAIN;
  e.bias = bias;
  e.out32 = out;
  e.ld_out = ld;
  return e;
}
EpiDesc epi_hidden(const float* bias, float* z, __nv_bfloat16* hb) {
  EpiDesc e{};
  e.mode = EPI_HIDDEN;
  e.bias = bias;
  e.out32 = z;
  e.ld_out = kMlpH;
  e.outb = hb;
  e.ld_outb = kMlpH;
  return e;
}
EpiDesc epi_back(const float* zin, float* g, __nv_bfloat16* gb) {
  EpiDesc e{};
  e.mode = EPI_BACK;
  e.zin = zin;
  e.ld_z = kMlpH;
  e.out32 = g;
  e.ld_out = kMlpH;
  e.outb = gb;
  e.ld_outb = kMlpH;
  return e;
}

}  // namespace

cudaError_t mlp_alloc(Mlp& M, int cap) {
  mlp_free(M);
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  A(dalloc(M.params, kMlpParams));
  A(dalloc(M.adam_m, kMlpParams));
  A(dalloc(M.adam_v, kMlpParams));
  A(dalloc(M.grad, kMlpParams));
  A(dalloc(M.step, 1));
  A(dalloc(M.w1b, kMlpInPad * kMlpH));
  A(dalloc(M.w2b, kMlpH * kMlpH));
  A(dalloc(M.w3b, kMlpH * kMlpOutPad));
  A(dalloc(M.xb, (size_t)cap * kMlpInPad));
  A(dalloc(M.z1, (size_t)cap * kMlpH));
  A(dalloc(M.h1b, (size_t)cap * kMlpH));
  A(dalloc(M.z2, (size_t)cap * kMlpH));
  A(dalloc(M.h2b, (size_t)cap * kMlpH));
  A(dalloc(M.out, (size_t)cap * kMlpOutPad));
  A(dalloc(M.dout, (size_t)cap * kMlpOutPad));
  A(dalloc(M.doutb, (size_t)cap * kMlpOutPad));
  A(dalloc(M.dz2, (size_t)cap * kMlpH));
  A(dalloc(M.dz2b, (size_t)cap * kMlpH));
  A(dalloc(M.dz1, (size_t)cap * kMlpH));
  A(dalloc(M.dz1b, (size_t)cap * kMlpH));
  A(dalloc(M.tdir, (size_t)cap * kMlpIn));
  A(dalloc(M.tls, (size_t)cap * kMlpIn));
  A(dalloc(M.nbr, (size_t)cap * kMaxNbr));
  A(dalloc(M.stats, 2 * kMlpIn + (size_t)cap * kMlpIn));  // mean, sd, then standardised coordinates
  A(dalloc(M.row_loss, cap));
  A(dalloc(M.loss, 1));
  A(dalloc(M.part, std::max((size_t)kMlpMaxSplit * kMlpH * kMlpH, (size_t)cap * kMlpH)));
  if (e == cudaSuccess) {
    // padded rows/columns of the weight copies and outputs stay zero
    A(cudaMemset(M.w1b, 0, sizeof(__nv_bfloat16) * kMlpInPad * kMlpH));
    A(cudaMemset(M.w3b, 0, sizeof(__nv_bfloat16) * kMlpH * kMlpOutPad));
    A(cudaMemset(M.out, 0, sizeof(float) * (size_t)cap * kMlpOutPad));
    A(cudaMemset(M.step, 0, sizeof(int)));
  }
  if (e != cudaSuccess) {
    mlp_free(M);
    return e;
  }
  M.cap = cap;
  return cudaSuccess;
}

void mlp_free(Mlp& M) {
  auto F = [](auto*& p) {
    if (p) cudaFree(p);
    p = nullptr;
  };
  F(M.params), F(M.adam_m), F(M.adam_v), F(M.grad), F(M.step), F(M.w1b), F(M.w2b), F(M.w3b), F(M.xb);
  F(M.z1), F(M.h1b), F(M.z2), F(M.h2b), F(M.out), F(M.dout), F(M.doutb), F(M.dz2), F(M.dz2b), F(M.dz1);
  F(M.dz1b), F(M.tdir), F(M.tls), F(M.nbr), F(M.stats), F(M.row_loss), F(M.loss), F(M.part);
  if (M.graph) cudaGraphExecDestroy(M.graph);
  M.graph = nullptr;
  M.graph_rows = M.graph_d = M.graph_nodes = 0;
  M.cap = 0;
}

static cudaError_t reset_adam(Mlp& M, cudaStream_t st, long long* L) {
  cudaError_t e = cudaMemsetAsync(M.adam_m, 0, sizeof(float) * kMlpParams, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(M.adam_v, 0, sizeof(float) * kMlpParams, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(M.step, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_mlp_bf16_weights<<<(kMlpParams + 255) / 256, 256, 0, st>>>(M.params, M.w1b, M.w2b, M.w3b);
  if (L) *L += 1;
  return cudaGetLastError();
}

cudaError_t mlp_init(Mlp& M, uint64_t seed, cudaStream_t st, long long* L) {
  k_mlp_init<<<(kMlpParams + 255) / 256, 256, 0, st>>>(M.params, (unsigned)(seed & 0xFFFFFFFFu),
                                                       (unsigned)(seed >> 32));
  if (L) *L += 1;
  const cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : reset_adam(M, st, L);
}

cudaError_t mlp_load(Mlp& M, const float* params_dev, cudaStream_t st, long long* L) {
  const cudaError_t e = cudaMemcpyAsync(M.params, params_dev, sizeof(float) * kMlpParams, cudaMemcpyDeviceToDevice, st);
  return e != cudaSuccess ? e : reset_adam(M, st, L);
}

cudaError_t mlp_targets(Mlp& M, const double* live_u, int n, int d, int k, cudaStream_t st, long long* L) {
  if (n > M.cap || d < 1 || d > kMlpIn || k < 1 || k > kMaxNbr || k >= n) return cudaErrorInvalidValue;
  double* xs = M.stats + 2 * kMlpIn;
  k_live_stats<<<1, 32 * kMlpIn, 0, st>>>(live_u, n, d, M.stats);
  k_standardise<<<(n * kMlpInPad + 255) / 256, 256, 0, st>>>(live_u, n, d, M.stats, xs, M.xb);
  k_local_pca<<<(n + kTargetWarps - 1) / kTargetWarps, 32 * kTargetWarps, 0, st>>>(live_u, xs, n, d, k, M.tdir, M.tls,
                                                                                  M.nbr);
  if (L) *L += 3;
  return cudaGetLastError();
}

cudaError_t mlp_inputs(Mlp& M, const float* x_std, int n, cudaStream_t st, long long* L) {
  if (n > M.cap) return cudaErrorInvalidValue;
  k_inputs_f32<<<(n * kMlpInPad + 255) / 256, 256, 0, st>>>(x_std, n, M.xb);
  if (L) *L += 1;
  return cudaGetLastError();
}

cudaError_t mlp_forward(Mlp& M, int n, cudaStream_t st, long long* L) {
  if (n > M.cap) return cudaErrorInvalidValue;
  cudaError_t e;
  e = gemm(M, M.xb, kMlpInPad, 1, M.w1b, kMlpH, 1, n, kMlpH, kMlpInPad,
           epi_hidden(M.params + kMlpOffB1, M.z1, M.h1b), st, L);
  if (e == cudaSuccess)
    e = gemm(M, M.h1b, kMlpH, 1, M.w2b, kMlpH, 1, n, kMlpH, kMlpH, epi_hidden(M.params + kMlpOffB2, M.z2, M.h2b), st, L);
  if (e == cudaSuccess)
    e = gemm(M, M.h2b, kMlpH, 1, M.w3b, kMlpOutPad, 1, n, kMlpOut, kMlpH,
             epi_plain(M.params + kMlpOffB3, M.out, kMlpOutPad), st, L);
  return e;
}

cudaError_t mlp_loss_grad(Mlp& M, int n, int d, cudaStream_t st, long long* L) {
  cudaError_t e = mlp_forward(M, n, st, L);
  if (e != cudaSuccess) return e;
  k_mlp_loss<<<(n + 127) / 128, 128, 0, st>>>(M.out, M.tdir, M.tls, n, d, M.dout, M.doutb, M.row_loss);
  k_mean<<<1, 256, 0, st>>>(M.row_loss, n, M.loss);
  if (L) *L += 2;
  // W3: H2^T dO;  dZ2 = (dO W3^T) silu'(Z2)
  e = gemm(M, M.h2b, 1, kMlpH, M.doutb, kMlpOutPad, 1, kMlpH, kMlpOut, n,
           epi_plain(nullptr, M.grad + kMlpOffW3, kMlpOut), st, L);
  if (e == cudaSuccess)
    e = gemm(M, M.doutb, kMlpOutPad, 1, M.w3b, 1, kMlpOutPad, n, kMlpH, kMlpOutPad, epi_back(M.z2, M.dz2, M.dz2b), st, L);
  // W2: H1^T dZ2;  dZ1 = (dZ2 W2^T) silu'(Z1)
  if (e == cudaSuccess)
    e = gemm(M, M.h1b, 1, kMlpH, M.dz2b, kMlpH, 1, kMlpH, kMlpH, n, epi_plain(nullptr, M.grad + kMlpOffW2, kMlpH), st, L);
  if (e == cudaSuccess)
    e = gemm(M, M.dz2b, kMlpH, 1, M.w2b, 1, kMlpH, n, kMlpH, kMlpH, epi_back(M.z1, M.dz1, M.dz1b), st, L);
  // W1: X^T dZ1
  if (e == cudaSuccess)
    e = gemm(M, M.xb, 1, kMlpInPad, M.dz1b, kMlpH, 1, kMlpIn, kMlpH, n, epi_plain(nullptr, M.grad + kMlpOffW1, kMlpH), st,
             L);
  if (e != cudaSuccess) return e;
  k_col_sum<<<1, 32, 0, st>>>(M.dout, n, kMlpOutPad, kMlpOut, M.grad + kMlpOffB3);
  k_col_sum<<<1, kMlpH, 0, st>>>(M.dz2, n, kMlpH, kMlpH, M.grad + kMlpOffB2);
  k_col_sum<<<1, kMlpH, 0, st>>>(M.dz1, n, kMlpH, kMlpH, M.grad + kMlpOffB1);
  if (L) *L += 3;
  return cudaGetLastError();
}

cudaError_t mlp_adam(Mlp& M, float lr, cudaStream_t st, long long* L) {
  k_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(M.params, M.grad, M.adam_m, M.adam_v, M.step, lr, M.w1b, M.w2b,
                                                   M.w3b);
  k_step_inc<<<1, 1, 0, st>>>(M.step);
  if (L) *L += 2;
  return cudaGetLastError();
}

cudaError_t mlp_train(Mlp& M, int n, int d, int steps, float lr, cudaStream_t st, long long* L) {
  if (steps <= 0) return cudaSuccess;
  if (!M.graph || M.graph_rows != n || M.graph_d != d || M.graph_lr != lr) {
    if (M.graph) cudaGraphExecDestroy(M.graph);
    M.graph = nullptr;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = mlp_loss_grad(M, n, d, cs, nullptr);
      if (e1 == cudaSuccess) e1 = mlp_adam(M, lr, cs, nullptr);
      e = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess) e = e1;
    }
    size_t nodes = 0;
    if (e == cudaSuccess) e = cudaGraphGetNodes(graph, nullptr, &nodes);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&M.graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      M.graph = nullptr;
      return e;
    }
    M.graph_rows = n;
    M.graph_d = d;
    M.graph_lr = lr;
    M.graph_nodes = (int)nodes;
  }
  for (int s = 0; s < steps; ++s) {
    const cudaError_t e = cudaGraphLaunch(M.graph, st);
    if (e != cudaSuccess) return e;
    if (L) *L += M.graph_nodes;
  }
  return cudaSuccess;
}

}  // namespace swig

// ---------------------------------------------------------------------------
// C-ABI: the network's pieces on host buffers (verification and tooling)
// ---------------------------------------------------------------------------
#include <string>
#include <vector>

#include "context.h"
#include "swig.h"

using namespace swig;

namespace {

int mfail(swig_ctx* c, int code, const std::string& m) {
  c->err = m;
  return code;
}

#define MCUDA(call)                                                                                         \
  do {                                                                                                      \
    cudaError_t e_ = (call);                                                                                \
    if (e_ != cudaSuccess)                                                                                  \
      return mfail(c, e_ == cudaErrorMemoryAllocation ? SWIG_E_NOMEM : SWIG_E_CUDA,                         \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                                     \
  } while (0)

// The context's network, with buffers for at least n rows.
int ensure_mlp(swig_ctx* c, int n) {
  if (n < 1 || n > 8192) return mfail(c, SWIG_E_ARG, "need 1 <= n <= 8192");
  MCUDA(cudaSetDevice(c->device));
  if (!c->mlp) c->mlp = new Mlp();
  if (c->mlp->cap < n) MCUDA(mlp_alloc(*c->mlp, std::max(n, 1024)));
  return SWIG_OK;
}

// Host parameters -> master weights (fresh Adam state and BF16 copies).
int upload_params(swig_ctx* c, const float* params) {
  float* tmp = nullptr;
  MCUDA(cudaMalloc(&tmp, sizeof(float) * kMlpParams));
  cudaError_t e = cudaMemcpy(tmp, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = mlp_load(*c->mlp, tmp, c->stream, &c->n_launches);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(tmp);
  MCUDA(e);
  c->h2d_bytes += sizeof(float) * kMlpParams;
  return SWIG_OK;
}

template <typename T>
int upload(swig_ctx* c, T* dst, const T* src, size_t n) {
  MCUDA(cudaMemcpy(dst, src, sizeof(T) * n, cudaMemcpyHostToDevice));
  c->h2d_bytes += sizeof(T) * n;
  return SWIG_OK;
}

// rows of a [n][ld] device array -> [n][w] host array
template <typename T>
int download_rows(swig_ctx* c, T* dst, const T* src, int n, int ld, int w) {
  std::vector<T> tmp((size_t)n * ld);
  MCUDA(cudaMemcpy(tmp.data(), src, sizeof(T) * tmp.size(), cudaMemcpyDeviceToHost));
  c->d2h_bytes += sizeof(T) * tmp.size();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < w; ++j) dst[(size_t)i * w + j] = tmp[(size_t)i * ld + j];
  return SWIG_OK;
}

}  // namespace

void swig_mlp_release(swig_ctx* c) {
  if (c && c->mlp) {
    mlp_free(*c->mlp);
    delete c->mlp;
    c->mlp = nullptr;
  }
}

extern "C" {

int swig_mlp_init(swig_ctx* c, uint64_t seed, float* params_out) {
  if (!c) return SWIG_E_ARG;
  if (!params_out) return mfail(c, SWIG_E_ARG, "null output");
  int rc = ensure_mlp(c, 1);
  if (rc) return rc;
  MCUDA(mlp_init(*c->mlp, seed, c->stream, &c->n_launches));
  MCUDA(cudaStreamSynchronize(c->stream));
  MCUDA(cudaMemcpy(params_out, c->mlp->params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  c->d2h_bytes += sizeof(float) * kMlpParams;
  return SWIG_OK;
}

int swig_mlp_forward(swig_ctx* c, const float* params, const float* x_std, int64_t n, float* out) {
  if (!c) return SWIG_E_ARG;
  if (!params || !x_std || !out) return mfail(c, SWIG_E_ARG, "null buffer");
  int rc = ensure_mlp(c, (int)std::min<int64_t>(n, 1 << 30));
  if (rc) return rc;
  if ((rc = upload_params(c, params))) return rc;
  float* xd = nullptr;
  MCUDA(cudaMalloc(&xd, sizeof(float) * n * kMlpIn));
  cudaError_t e = cudaMemcpy(xd, x_std, sizeof(float) * n * kMlpIn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = mlp_inputs(*c->mlp, xd, (int)n, c->stream, &c->n_launches);
  if (e == cudaSuccess) e = mlp_forward(*c->mlp, (int)n, c->stream, &c->n_launches);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(xd);
  MCUDA(e);
  c->h2d_bytes += sizeof(float) * n * kMlpIn;
  return download_rows(c, out, c->mlp->out, (int)n, kMlpOutPad, kMlpOut);
}

int swig_mlp_loss_grad(swig_ctx* c, const float* params, const float* x_std, const float* tdir, const float* tls,
                       int64_t n, int d, double* loss_out, float* grad_out) {
  if (!c) return SWIG_E_ARG;
  if (!params || !x_std || !tdir || !tls || !loss_out || !grad_out) return mfail(c, SWIG_E_ARG, "null buffer");
  if (d < 1 || d > kMlpIn) return mfail(c, SWIG_E_ARG, "need 1 <= d <= 13");
  int rc = ensure_mlp(c, (int)std::min<int64_t>(n, 1 << 30));
  if (rc) return rc;
  if ((rc = upload_params(c, params))) return rc;
  Mlp& M = *c->mlp;
  if ((rc = upload(c, M.tdir, tdir, (size_t)n * kMlpIn))) return rc;
  if ((rc = upload(c, M.tls, tls, (size_t)n * kMlpIn))) return rc;
  float* xd = nullptr;
  MCUDA(cudaMalloc(&xd, sizeof(float) * n * kMlpIn));
  cudaError_t e = cudaMemcpy(xd, x_std, sizeof(float) * n * kMlpIn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = mlp_inputs(M, xd, (int)n, c->stream, &c->n_launches);
  if (e == cudaSuccess) e = mlp_loss_grad(M, (int)n, d, c->stream, &c->n_launches);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(xd);
  MCUDA(e);
  c->h2d_bytes += sizeof(float) * n * kMlpIn;
  MCUDA(cudaMemcpy(loss_out, M.loss, sizeof(double), cudaMemcpyDeviceToHost));
  MCUDA(cudaMemcpy(grad_out, M.grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  c->d2h_bytes += sizeof(double) + sizeof(float) * kMlpParams;
  return SWIG_OK;
}

int swig_mlp_targets(swig_ctx* c, const double* live_u, int64_t n, int d, float* tdir, float* tls, int* nbr) {
  if (!c) return SWIG_E_ARG;
  if (!live_u || !tdir || !tls) return mfail(c, SWIG_E_ARG, "null buffer");
  if (d < 1 || d > kMlpIn || 2 * d >= n) return mfail(c, SWIG_E_ARG, "need 1 <= d <= 13 and 2d < n");
  int rc = ensure_mlp(c, (int)std::min<int64_t>(n, 1 << 30));
  if (rc) return rc;
  Mlp& M = *c->mlp;
  double* ud = nullptr;
  MCUDA(cudaMalloc(&ud, sizeof(double) * n * d));
  cudaError_t e = cudaMemcpy(ud, live_u, sizeof(double) * n * d, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = mlp_targets(M, ud, (int)n, d, 2 * d, c->stream, &c->n_launches);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(ud);
  MCUDA(e);
  c->h2d_bytes += sizeof(double) * n * d;
  if ((rc = download_rows(c, tdir, M.tdir, (int)n, kMlpIn, kMlpIn))) return rc;
  if ((rc = download_rows(c, tls, M.tls, (int)n, kMlpIn, kMlpIn))) return rc;
  if (nbr && (rc = download_rows(c, nbr, M.nbr, (int)n, 2 * kMlpIn, 2 * kMlpIn))) return rc;
  return SWIG_OK;
}

int swig_mlp_train(swig_ctx* c, const double* live_u, int64_t n, int d, int steps, double lr, float* params_inout,
                   float* out_rows) {
  if (!c) return SWIG_E_ARG;
  if (!live_u || !params_inout) return mfail(c, SWIG_E_ARG, "null buffer");
  if (d < 1 || d > kMlpIn || 2 * d >= n) return mfail(c, SWIG_E_ARG, "need 1 <= d <= 13 and 2d < n");
  if (steps < 0 || !(lr > 0.0)) return mfail(c, SWIG_E_ARG, "need steps >= 0 and lr > 0");
  int rc = ensure_mlp(c, (int)std::min<int64_t>(n, 1 << 30));
  if (rc) return rc;
  if ((rc = upload_params(c, params_inout))) return rc;
  Mlp& M = *c->mlp;
  double* ud = nullptr;
  MCUDA(cudaMalloc(&ud, sizeof(double) * n * d));
  cudaError_t e = cudaMemcpy(ud, live_u, sizeof(double) * n * d, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = mlp_targets(M, ud, (int)n, d, 2 * d, c->stream, &c->n_launches);
  if (e == cudaSuccess) e = mlp_train(M, (int)n, d, steps, (float)lr, c->stream, &c->n_launches);
  if (e == cudaSuccess && out_rows) e = mlp_forward(M, (int)n, c->stream, &c->n_launches);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(ud);
  MCUDA(e);
  c->h2d_bytes += sizeof(double) * n * d;
  MCUDA(cudaMemcpy(params_inout, M.params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  c->d2h_bytes += sizeof(float) * kMlpParams;
  if (out_rows && (rc = download_rows(c, out_rows, M.out, (int)n, kMlpOutPad, kMlpOut))) return rc;
  return SWIG_OK;
}

}  // extern "C"
