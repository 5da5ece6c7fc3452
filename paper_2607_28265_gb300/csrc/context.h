// The opaque swig_ctx behind the C-ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "kernels.h"
#include "swig.h"
#include "swig_internal.h"

namespace swig {
struct SamplerState;  // device state of a nested-sampling run (sampler.cu)
struct Mlp;           // learned-proposal network (mlp.cu)
}

struct swig_ctx {
  int device = 0;
  int sm_count = 1;
  cudaStream_t stream = nullptr;
  std::string err;
  // grid (Sec. 3.1): f_k = k df, k_min .. k_min + n_bins - 1
  double f_min = 0.0, f_max = 0.0, df = 0.0;
  int64_t k_min = 0, n_bins = 0;
  bool grid_set = false;
  // detectors
  bool det_set[SWIG_MAX_DET] = {false, false, false, false};
  double vertex[SWIG_MAX_DET][3] = {}, xarm[SWIG_MAX_DET][3] = {}, yarm[SWIG_MAX_DET][3] = {};
  double gmst = 0.0;
  std::vector<double> data[SWIG_MAX_DET], psd[SWIG_MAX_DET];
  // prior and sampler
  swig_param params[SWIG_N_PARAMS] = {};
  bool prior_set = false;
  int sky_a = -1, sky_b = -1;  // detector-frame sky parameterisation (baseline b -> a), -1: equatorial
  int n_sampled = 0;
  swig_sampler_cfg cfg = {};
  bool cfg_set = false;
  // prepared device state
  bool dirty = true;
  int prepared_precision = -1;
  int prepared_like = SWIG_LIKE_FULL;
  swig::LikeConst L = {};
  swig::DeviceBuffers B;
  swig::SamplerState* sampler = nullptr;
  swig::Mlp* mlp = nullptr;
  long long wait_limit = 10000000;  // spins of a bounded device wait (~100 ns each)
  // results of the last run
  swig_result last = {};
  double profile[25] = {};
  std::vector<double> cta_profile;  // [n_ctas][4] of the last run (see swig_get_profile)
  // counters over the context's lifetime: kernel launches, bytes copied host
  // to device and device to host by the library
  long long n_launches = 0, h2d_bytes = 0, d2h_bytes = 0;
  bool own_stream = true;
  std::vector<double> out_theta, out_logl, out_logw;
};

namespace swig {
int prepare(swig_ctx* c);
int ensure_scratch(swig_ctx* c, int n);
int loglike_device(swig_ctx* c, const double* theta_dev, int64_t n, double* out_dev, cudaStream_t st);
int current_precision(const swig_ctx* c);
// The sky frame of the context (on = 0 when equatorial); SWIG_OK or a status
// with the context's error set when the prior does not fit the frame.
int make_sky_frame(swig_ctx* c, SkyFrame* out);
}  // namespace swig

void swig_sampler_release(swig_ctx* c);
void swig_mlp_release(swig_ctx* c);
