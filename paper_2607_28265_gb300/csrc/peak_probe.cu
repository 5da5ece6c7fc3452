// Throughput of the special-function unit on this GPU: __sincosf (one sine
// and one cosine result per call, the per-bin operation of the likelihood's
// inner loop) and, for comparison, FP32 FFMA, per SM per clock at the
// device's maximum clock.  A standalone program (not part of libswig): the
// bench compiles and runs it to take the roofline denominator of the
// SFU-bound sweep from a measurement on the same GPU.
//
// Each thread runs `rounds` rounds over 8 independent values (4 CTAs of 512
// threads per SM, 64 warps); the best of 5 launches is reported.  Every read
// and write is in bounds (one float per thread).  Output: one JSON line per
// kind.
#include <cuda_runtime.h>

#include <cstdio>

__global__ void k_sincos(float* out, int rounds, float step) {
  float v[8], a = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = 0.01f * (float)(threadIdx.x + j);
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float s, c;
      __sincosf(v[j], &s, &c);
      v[j] = s + c * step;  // bounded argument, a dependence between rounds
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) a += v[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = a;
}

__global__ void k_ffma(float* out, int rounds, float step) {
  float v[8], a = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = 0.01f * (float)(threadIdx.x + j);
  for (int r = 0; r < rounds; ++r) {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = fmaf(v[j], step, 0.5f);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) a += v[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = a;
}

int main() {
  int dev = 0, sms = 0, clk_khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int threads = 512, blocks = sms * 4, rounds = 4096;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * threads * blocks) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int which = 0; which < 2; ++which) {
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
      cudaEventRecord(e0);
      if (which == 0)
        k_sincos<<<blocks, threads>>>(out, rounds, 0.37f);
      else
        k_ffma<<<blocks, threads>>>(out, rounds, 0.999f);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) return 2;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    const double n_ops = (double)threads * blocks * rounds * 8 * (which == 0 ? 2 : 1);
    const double per_s = n_ops / (best * 1e-3);
    std::printf("{\"kind\": \"%s\", \"ms\": %.4f, \"ops_per_s\": %.6e, \"per_clk_per_sm_at_max_clock\": %.4f, "
                "\"sms\": %d, \"max_clock_khz\": %d}\n",
                which == 0 ? "sfu_sincos_results" : "ffma", best, per_s, per_s / ((double)sms * clk_khz * 1e3), sms,
                clk_khz);
  }
  cudaFree(out);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
