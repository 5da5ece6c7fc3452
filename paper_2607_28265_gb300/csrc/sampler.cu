// Nested sampling driver (filled in with the persistent SwiG kernel).
#include <cuda_runtime.h>

#include "context.h"
#include "swig.h"

void swig_sampler_release(swig_ctx* c) { (void)c; }

extern "C" {
int swig_run(swig_ctx* c, swig_result* out) {
  if (!c) return SWIG_E_ARG;
  (void)out;
  c->err = "nested sampling not built yet";
  return SWIG_E_STATE;
}
int swig_get_samples(swig_ctx* c, double* theta, double* logl, double* logw, int64_t cap, int64_t* n_out) {
  if (!c) return SWIG_E_ARG;
  (void)theta; (void)logl; (void)logw; (void)cap;
  if (n_out) *n_out = 0;
  return SWIG_OK;
}
}
