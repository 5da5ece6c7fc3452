// Learned slice proposal: a 13 -> 256 -> 256 -> 26 SiLU network trained on the
// sampler's own live points (device side).
//
// The paper draws slice directions from the live covariance (Sec. 2.3, Eq. 3;
// Sec. 3.2); this network is the library's optional alternative.  Per live
// point it predicts a direction u and log-widths s; a chain's slice direction
// for Gibbs block b is exp(s_b) * u_b / |u_b| from the row of a live point
// drawn uniformly from a frozen snapshot, so the move does not depend on the
// chain's position and the slice kernel stays exact.  Training targets are the
// local principal direction (correlation matrix of the 2d nearest live
// neighbours) and the neighbours' log standard deviations.
//
// Arithmetic: every matrix-product operand is bfloat16 (inputs, activations,
// output gradients, weight copies), accumulation FP32 on the tensor cores
// (mma.sync m16n8k16), biases/SiLU/loss FP32, master weights and Adam FP32.
// Parameter layout (FP32, flat): W1 [13][256], b1 [256], W2 [256][256],
// b2 [256], W3 [256][26], b3 [26], row index = input unit.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace swig {

constexpr int kMlpIn = 13, kMlpInPad = 16, kMlpH = 256, kMlpOut = 26, kMlpOutPad = 32;
constexpr int kMlpOffW1 = 0;
constexpr int kMlpOffB1 = kMlpOffW1 + kMlpIn * kMlpH;
constexpr int kMlpOffW2 = kMlpOffB1 + kMlpH;
constexpr int kMlpOffB2 = kMlpOffW2 + kMlpH * kMlpH;
constexpr int kMlpOffW3 = kMlpOffB2 + kMlpH;
constexpr int kMlpOffB3 = kMlpOffW3 + kMlpH * kMlpOut;
constexpr int kMlpParams = kMlpOffB3 + kMlpOut;  // 76,058
constexpr int kMlpMaxSplit = 8;                  // split-K partial buffers

struct Mlp {
  int cap = 0;  // rows (live points) the buffers hold
  float* params = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* grad = nullptr;
  int* step = nullptr;  // Adam step counter
  __nv_bfloat16* w1b = nullptr;  // [16][256], rows 13..15 zero
  __nv_bfloat16* w2b = nullptr;  // [256][256]
  __nv_bfloat16* w3b = nullptr;  // [256][32], columns 26..31 zero
  __nv_bfloat16* xb = nullptr;   // [cap][16] standardised inputs
  float* z1 = nullptr;           // [cap][256]
  __nv_bfloat16* h1b = nullptr;
  float* z2 = nullptr;
  __nv_bfloat16* h2b = nullptr;
  float* out = nullptr;           // [cap][32]
  float* dout = nullptr;          // [cap][32]
  __nv_bfloat16* doutb = nullptr;
  float* dz2 = nullptr;           // [cap][256]
  __nv_bfloat16* dz2b = nullptr;
  float* dz1 = nullptr;
  __nv_bfloat16* dz1b = nullptr;
  float* tdir = nullptr;          // [cap][13]
  float* tls = nullptr;           // [cap][13]
  int* nbr = nullptr;             // [cap][26] neighbour indices
  double* stats = nullptr;        // mean[13], sd[13]
  double* row_loss = nullptr;     // [cap]
  double* loss = nullptr;         // [1]
  float* part = nullptr;          // [kMlpMaxSplit][256][256] split-K partials
  cudaGraphExec_t graph = nullptr;  // one training step for (graph_rows, graph_d)
  int graph_rows = 0, graph_d = 0, graph_nodes = 0;
  float graph_lr = 0.0f;
};

cudaError_t mlp_alloc(Mlp& M, int cap);
void mlp_free(Mlp& M);
// Philox-4x32-10 initial weights N(0, 1/fan_in), biases 0; resets Adam.
cudaError_t mlp_init(Mlp& M, uint64_t seed, cudaStream_t st, long long* launches);
// Copy FP32 parameters (device pointer) into the master weights; resets Adam.
cudaError_t mlp_load(Mlp& M, const float* params_dev, cudaStream_t st, long long* launches);
// Standardised inputs and training targets of n live points (device, n x d doubles).
cudaError_t mlp_targets(Mlp& M, const double* live_u, int n, int d, int k, cudaStream_t st, long long* launches);
// Standardised inputs given directly (device, n x 13 floats).
cudaError_t mlp_inputs(Mlp& M, const float* x_std, int n, cudaStream_t st, long long* launches);
// Output rows of n points into M.out.
cudaError_t mlp_forward(Mlp& M, int n, cudaStream_t st, long long* launches);
// Forward, loss and parameter gradient into M.grad (loss in M.loss).
cudaError_t mlp_loss_grad(Mlp& M, int n, int d, cudaStream_t st, long long* launches);
// One Adam step on M.grad (step counter on the device).
cudaError_t mlp_adam(Mlp& M, float lr, cudaStream_t st, long long* launches);
// `steps` training steps (loss_grad + adam) replayed from a captured graph.
cudaError_t mlp_train(Mlp& M, int n, int d, int steps, float lr, cudaStream_t st, long long* launches);

}  // namespace swig
