// Batched likelihood that allocates no memory: the per-call scratch lives in
// a fixed array in the library's device image instead of buffers obtained with
// cudaMalloc.
//
// Who needs this: code that must not allocate device memory while it runs --
// a caller inside a real-time or latency-critical loop that has pre-reserved
// all of its memory, an allocator-free embedding (a host runtime that forbids
// cudaMalloc/cudaFree after start-up, or that records its work into a graph and
// cannot let the library allocate behind its back), or a process whose memory
// pool is owned by another framework.  Such callers prepare the context once
// (which does allocate), then call this entry point as often as they like.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "context.h"
#include "kernels.h"
#include "swig.h"

namespace swig {

// 8 MiB of scratch, reserved on every device that loads the library for as
// long as the process runs.
constexpr size_t kNoAllocScratchBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

size_t round_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Device address of the scratch array on `device` (set-up on first use, with
// that device current).  The array's host-side name is only a stand-in and
// must never be handed to a kernel.
cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return cudaSuccess;
}

}  // namespace
}  // namespace swig

using namespace swig;

extern "C" int swig_loglike_batch_noalloc(swig_ctx* c, const double* theta_dev, int64_t n, double* out_logl_dev,
                                          void* stream) {
  if (!c) return SWIG_E_ARG;
  if (n == 0) return SWIG_OK;
  if (n < 0 || !theta_dev || !out_logl_dev) {
    c->err = "need n >= 0 and non-null device buffers";
    return SWIG_E_ARG;
  }
  if (c->dirty || c->prepared_precision != SWIG_PREC_MIXED || c->prepared_like != SWIG_LIKE_FULL) {
    c->err = "the context must be prepared for the mixed-precision full-grid likelihood by an earlier swig_loglike_batch(_dev) or "
             "swig_run call with the current problem (preparation allocates; this entry point does not)";
    return SWIG_E_STATE;
  }
  // Capacity first, from the per-vector bytes (three 256-byte roundings at
  // most on top), so that no size below is formed from an unchecked n.
  const size_t per_theta = sizeof(EvalRecord) + sizeof(float) * kAnchorStride * (size_t)c->L.n_tiles +
                           sizeof(float) * kPartialStride * (size_t)c->L.n_slices * 4;
  const int64_t cap = (int64_t)((kNoAllocScratchBytes - 3 * 256) / per_theta);
  if (n > cap) {
    c->err = "batch of " + std::to_string(n) + " exceeds the fixed scratch of this entry point (" +
             std::to_string(kNoAllocScratchBytes >> 20) + " MiB, " + std::to_string(cap) +
             " parameter vectors for this grid); split the batch";
    return SWIG_E_ARG;
  }
  // layout: [records][anchors][partials], each 256-byte aligned
  const size_t rec_b = round_up(sizeof(EvalRecord) * (size_t)n);
  const size_t anc_b = round_up(sizeof(float) * kAnchorStride * (size_t)c->L.n_tiles * (size_t)n);
  cudaError_t e = cudaSetDevice(c->device);
  void* base = nullptr;
  if (e == cudaSuccess) e = scratch_address(c->device, &base);
  if (e != cudaSuccess) {
    c->err = std::string("scratch set-up: ") + cudaGetErrorString(e);
    return SWIG_E_CUDA;
  }
  // Every scratch word this call reads is written earlier in the same call
  // (records, anchors, one partial per work unit), so nothing needs clearing.
  DeviceBuffers B = c->B;
  unsigned char* p = static_cast<unsigned char*>(base);
  B.rec = reinterpret_cast<EvalRecord*>(p);
  B.anchors = reinterpret_cast<float*>(p + rec_b);
  B.partials32 = reinterpret_cast<float*>(p + rec_b + anc_b);
  B.cap = (int)n;
  e = launch_loglike_mixed(c->L, B, theta_dev, (int)n, out_logl_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    c->err = std::string("likelihood launch: ") + cudaGetErrorString(e);
    return SWIG_E_CUDA;
  }
  c->n_launches += 4;
  return SWIG_OK;
}
