// Persistent Slice-within-Gibbs nested sampler (Sec. 2.2, 2.3, 3.2 of the paper).
//
// One cooperative launch runs up to `max_iters` nested-sampling iterations on
// the device.  Every CTA owns one slice of the frequency grid (its data staged
// once in shared memory).  The grid meets at a barrier only around the
// iteration boundary:
//
//   boundary  (CTA 0, once per NS iteration): write the k finished chains back
//             into the live set, sort the live log-likelihoods, test the
//             termination rule log Z_live - log Z_dead < dlogz, retire the k
//             worst points into the dead buffer with weights L_j (X_{j-1} - X_j)
//             (log X shrinks by 1/n per death, n = m, m-1, ..., m-k+1), set
//             logL* to the lowest survivor, estimate the live covariance and
//             its per-block Cholesky factors, and start k chains at survivors.
//
// Within the iteration everything runs as a dataflow (k_ns_flow):
//
//   control   (warp 0 of the chain's home CTA): advance the chain's hit-and-run
//             slice state machine (Neal 2003 stepping-out and shrinkage along a
//             direction drawn from the block covariance, or a learned one)
//             through every proposal that needs no pass over the grid:
//             proposals outside the unit cube, and proposals of blocks that only
//             change the projection factors C_i (d_L, iota, psi, phi_c), which
//             reuse the chain's cached per-detector sums kappa_i.  A proposal
//             that changes the waveform or the time shifts is set up (one lane
//             per piece of the record) and published as a request.
//   sweep     (warps 1.. of every CTA): claim published requests and evaluate
//             the CTA's slice for them, one warp per (chain, slice), partial
//             sums per (chain, slice); the chain's control resumes when every
//             CTA has counted itself done.
//
// Every spin-wait is bounded; on expiry the kernel records SWIG_E_TIMEOUT and
// every CTA returns at its next barrier.  The heterodyned likelihood has its
// own persistent kernel (k_ns_het, one CTA per chain).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"
#include "het.cuh"
#include "mlp.h"
#include "sweep.cuh"

namespace swig {

constexpr int kMaxDim = SWIG_N_PARAMS;
constexpr int kMaxBlocks = 16;
constexpr int kMaxStepOut = 100;
constexpr int kMaxShrink = 100;
constexpr int kMaxSort = 8192;
constexpr int kMaxChains = 2048;

constexpr int kMaxEvents = 4;    // events per multi-event launch
constexpr int kFlowThreads = 512;  // dataflow sampler: 16 warps, up to 128 registers per thread
constexpr int kHetThreads = 512;  // heterodyned sampler: one chain per CTA, 16 warps
static_assert(kHetThreads == kHetTmThreads, "the sampler and the batched time-marginalised kernel share sum orders");
constexpr int kFreeBudget = 8;  // projection-only evaluations per chain per round
#ifndef SWIG_FLOW_PARTS
#define SWIG_FLOW_PARTS 1
#endif
static_assert(SWIG_FLOW_PARTS >= 1 && SWIG_FLOW_PARTS <= 4, "1..4 parts per slice");
// 1: both ends of a bracket step out at once in the full-grid dataflow kernel
// (same evaluations and results as one end after the other, two requests in
// flight per chain); 0: one end at a time
#ifndef SWIG_PAR_OUT
#define SWIG_PAR_OUT 1
#endif
// Bytes of a slice's tile table plus `warps` anchor rows in the dataflow
// kernel's shared memory (16-byte aligned).
__host__ __device__ inline size_t flow_tile_bytes(int max_tiles, int warps) {
  const size_t ti = ((size_t)max_tiles * sizeof(TileInfo) + 15) & ~(size_t)15;
  return ti + (((size_t)warps * max_tiles * kAnchorStride * sizeof(float) + 15) & ~(size_t)15);
}
// PH_OUT: both ends of the bracket stepping out at once (two requests in flight)
enum ChainPhase { PH_NEW = 0, PH_LEFT = 1, PH_RIGHT = 2, PH_SHRINK = 3, PH_OUT = 4 };
// What a Gibbs block moves: waveform coefficients, amplitude A(Mc)/d_L,
// projection P_i, time shifts tau_i (BF_SKY: through the geocentric delays;
// BF_TAU alone: t_c).
enum BlockFlag { BF_INTR = 1, BF_AMP = 2, BF_PROJ = 4, BF_TAU = 8, BF_SPIN = 16, BF_TIDE = 32, BF_SKY = 64 };
enum RunStatus { ST_RUNNING = 0, ST_TERMINATED = 1, ST_LIMIT = 2 };

struct SamplerConst {
  int ndim, nlive, nrep, sweeps, steps_per_dim, n_blocks;
  int slot_of_dim[kMaxDim];
  int block_size[kMaxBlocks], block_free[kMaxBlocks], block_flags[kMaxBlocks];
  int block_dims[kMaxBlocks][kMaxDim];
  PriorSlot prior[SWIG_N_PARAMS];
  unsigned key0, key1;
  double dlogz;
  int m_pow2;
  int max_iters;
  long long spin_limit;
  int max_pieces;      // pieces per slice (sweep work units)
  int max_tiles_slice; // tiles overlapping the largest slice
  int n_ctas;
  int mixed;
  int flow_parts;   // parts per slice (dataflow kernel): fixed summation partition
  int het;          // heterodyned likelihood (projection-only evaluations use ChainState::vv)
  SkyFrame sky;     // detector-frame sky parameterisation (slots 9, 10), or off
  int learn_on;     // learned directions available (SWIG_PROPOSAL_LEARNED)
  float learn_mix;  // probability of a learned direction per slice step
  // warp-parallel control: dimensions of each block as a bit mask, each
  // dimension's rank within its block, the dimension of each slot (-1: none),
  // and the byte offset of the homed chains' state in dynamic shared memory
  unsigned block_mask[kMaxBlocks];
  int block_rank[kMaxDim];
  int dim_of_slot[SWIG_N_PARAMS];
  int ctl_off;
  int ctl_slots;  // chains homed per CTA at most
  // parallel stepping-out (full-grid dataflow kernel): the left end of a
  // chain's bracket uses request slot c, the right end slot nrep + c
  int par_out;
  int n_slots;    // request slots: nrep, or 2 nrep with par_out
  int claim_off;  // byte offset (in the dynamic shared memory after the slice data) of the claim words
                  // (heterodyned sampler: of the chunk anchors)
  int stage_off;  // heterodyned sampler: byte offset of the warps' chunk-table stages (0: none)
};

struct ChainState {
  double x[kMaxDim], y[kMaxDim], dir[kMaxDim];
  double th[SWIG_N_PARAMS], th_y[SWIG_N_PARAMS];  // theta of x and of the proposal
  double lx, lo, hi, t;
  double kap[2 * SWIG_MAX_DET];
  double vv[SWIG_MAX_DET];  // heterodyned path: <h|h>_i / |C_i|^2 of the current point, times A1^2
  int block, step, sweep, phase, n_out, n_shrink;
  int pending, done, proj_dirty, slot;
  unsigned ctr;
  int n_caps;
  long long n_evals, n_full;
  int side;     // PH_OUT: bit 0 the left end still stepping, bit 1 the right end
  int n_out_r;  // PH_OUT: expansions of the right end
};

struct NSGlobal {
  double logx, logz, logl_star;
  long long iter;
  int iters_launch;
  int status;
  int error;
  int chains_done;
  int need_writeback;
  int n_dead;
  unsigned bar_count, bar_gen;
  // phase timers of CTA 0 [ns, %globaltimer]: boundary, control, wait after
  // control, sweep, wait after sweep; and rounds
  unsigned long long t_bound, t_ctrl, t_wait_ctrl, t_sweep, t_wait_sweep, rounds;
  // chain 0's control breakdown [clock64 cycles]: pending result, new step,
  // proposal + transform, projection-only evaluations, full setup; counts
  unsigned long long c_result, c_step, c_prop, c_free, c_setup, n_free, n_setup, n_step;
  // CTA 0's sweep warps (dataflow kernel): units evaluated, clock64 cycles in
  // units, cycles idle (polling for work)
  unsigned long long f_units, f_unit_cyc, f_idle_cyc;
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct SamplerPtrs {
  double* live_u;      // [m][ndim]
  double* live_logl;   // [m]
  double* live_kap;    // [m][8]
  double* live_vv;     // [m][4] heterodyned path: see ChainState::vv
  ChainState* chains;  // [k]
  EvalRecord* recx;    // [k] setup record of each chain's current point
  int* pending;        // [k]
  float* chol;         // [kMaxBlocks][kMaxDim][kMaxDim]
  NSGlobal* g;
  double* dead_u;      // [max_iters * k][ndim]
  double* dead_logl;
  double* dead_logw;
  const double* harm;  // [k + 1]: sum_{i<j} 1 / (m - i)
  const double* lw;    // [m + 1]: log(1 - exp(-1/n))
  const int* piece_begin;  // [n_pieces_total + n_slices] absolute first bin of each piece, per slice
  const int* slice_piece;  // [n_slices + 1] offset of each slice's pieces in piece_begin
  float* anchor_buf;       // [n_slices][k][max_tiles_slice][kAnchorStride] per-round anchors
  const float* learn_out;  // [m][32] network outputs (u, s) of a frozen live snapshot, or null
  int* req;                // [k] 8 * (sequence number of the chain's latest full-likelihood request) + parts per slice
  int* done_cnt;           // [k] CTAs that finished the chain's latest request
  unsigned long long* cta_prof;  // [n_ctas][4] per CTA: sweep units, cycles in units, cycles polling, control cycles
};

// ---------------------------------------------------------------------------
// Draws built on Philox-4x32-10 (device_common.cuh).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double u01_from(uint4 r) {  // 53-bit uniform in [0, 1)
  return ((double)(r.x >> 5) * 67108864.0 + (double)(r.y >> 6)) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double chain_uniform(const SamplerConst& S, ChainState& ch, int c, long long it) {
  return u01_from(philox4x32_10(make_uint4(ch.ctr++, (unsigned)c, (unsigned)it, 0u), S.key0, S.key1));
}

// Standard normal by Box-Muller from one Philox block.
__device__ __forceinline__ float chain_normal(const SamplerConst& S, ChainState& ch, int c, long long it) {
  const uint4 r = philox4x32_10(make_uint4(ch.ctr++, (unsigned)c, (unsigned)it, 0u), S.key0, S.key1);
  const float u1 = ((float)(r.x >> 8) + 1.0f) * (1.0f / 16777216.0f);  // (0, 1]
  const float u2 = (float)(r.y >> 8) * (1.0f / 16777216.0f);
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// ---------------------------------------------------------------------------
// Bounded grid barrier (all CTAs co-resident by cooperative launch).
// ---------------------------------------------------------------------------
__device__ bool grid_sync(NSGlobal* g, int n_ctas, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &g->bar_gen;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&g->bar_count, 1u) + 1u;
    if (arrived == (unsigned)n_ctas) {
      atomicExch(&g->bar_count, 0u);
      __threadfence();
      atomicAdd(&g->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (++spins > limit) {
          atomicCAS(&g->error, 0, SWIG_E_TIMEOUT);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = (*(volatile int*)&g->error) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// Projection-only setup and FP32 epilogue for blocks that leave kappa unchanged.
// ---------------------------------------------------------------------------
__device__ inline void projection_record(const LikeConst& L, const double* th, EvalRecord* rec) {
  const double mc = th[0], dl = th[6], iota = th[7], psi = th[8], ra = th[9], dec = th[10], phic = th[12];
  rec->valid = (mc > 0.0 && dl > 0.0 && th[1] > 0.0 && th[1] <= 1.0) ? 1 : 0;
  const double amp = rec->valid ? amplitude_per_mpc(mc) / dl : 0.0;
  const double ci = cos(iota);
  const double plus = 0.5 * (1.0 + ci * ci), cross = -ci;
  double sph = 0.0, cph = 1.0;
  if (!L.phase_marg) sincos(phic, &sph, &cph);
  double hh = 0.0;
  for (int i = 0; i < L.n_det; ++i) {
    double fp, fx;
    antenna_fp_fx(L.dten[i], ra, dec, psi, L.gmst, &fp, &fx);
    const double re0 = amp * fp * plus, im0 = amp * fx * cross;
    rec->cre[i] = re0 * cph - im0 * sph;
    rec->cim[i] = re0 * sph + im0 * cph;
    hh += (rec->cre[i] * rec->cre[i] + rec->cim[i] * rec->cim[i]) * L.K[i];
  }
  rec->hh = hh;
}

// FP32 form of the same projection and epilogue (mixed precision): relative
// error ~1e-6 on |Z| and <h|h>, far inside the likelihood tolerance; the large
// constant -<d|d>/2 is added in FP64.
__device__ inline float log_i0_f32(float x) {
  if (x < 20.0f) {
    const float y = 0.25f * x * x;
    float term = 1.0f, sum = 1.0f;
    for (int k = 1; k < 64; ++k) {
      term *= y / (float)(k * k);
      sum += term;
      if (term < 1e-8f * sum) break;
    }
    return logf(sum);
  }
  const float t = 1.0f / (8.0f * x);
  const float s = 1.0f + t * (1.0f + t * (4.5f + t * (37.5f + t * 459.375f)));
  return x - 0.5f * logf(6.283185307179586f * x) + logf(s);
}

// kap: per-detector sums cached at the chain's current point (full grid:
// kappa_i; heterodyned: (Z_i / C_i) / inv_scale_i); vv (heterodyned only):
// <h|h>_i / |C_i|^2 times A1^2, replacing the constant K_i A1^2 of the full grid.
__device__ inline double free_loglike_mixed(const LikeConst& L, const double* th, const double* kap,
                                            const double* vv = nullptr) {
  const float mc = (float)th[0], dl = (float)th[6], iota = (float)th[7], psi = (float)th[8];
  const float ra = (float)th[9], dec = (float)th[10], phic = (float)th[12];
  if (!(mc > 0.0f && dl > 0.0f)) return -INFINITY;
  const float rel = exp2f(0.8333333333f * log2f(mc)) / dl;  // Mc^(5/6) / d_L
  float sl, cl, sd, cd, sp, cp;
  sincosf(ra - (float)L.gmst, &sl, &cl);
  sincosf(dec, &sd, &cd);
  sincosf(psi, &sp, &cp);
  const float east[3] = {-sl, cl, 0.0f};
  const float north[3] = {-sd * cl, -sd * sl, cd};
  float X[3], Y[3];
  for (int k = 0; k < 3; ++k) {
    X[k] = -cp * east[k] + sp * north[k];
    Y[k] = sp * east[k] + cp * north[k];
  }
  const float ci = cosf(iota);
  const float plus = 0.5f * (1.0f + ci * ci), cross = -ci;
  float sph = 0.0f, cph = 1.0f;
  if (!L.phase_marg) sincosf(phic, &sph, &cph);
  float zr = 0.0f, zi = 0.0f, hh = 0.0f;
  for (int i = 0; i < L.n_det; ++i) {
    float d[6];
    for (int q = 0; q < 6; ++q) d[q] = (float)L.dten[i][q];
    auto form = [&d](const float* a, const float* b) {
      return a[0] * (d[0] * b[0] + d[1] * b[1] + d[2] * b[2]) + a[1] * (d[1] * b[0] + d[3] * b[1] + d[4] * b[2]) +
             a[2] * (d[2] * b[0] + d[4] * b[1] + d[5] * b[2]);
    };
    const float fp = form(X, X) - form(Y, Y), fx = 2.0f * form(X, Y);
    const float re0 = rel * fp * plus, im0 = rel * fx * cross;
    const float cre = re0 * cph - im0 * sph, cim = re0 * sph + im0 * cph;
    const float a = (float)kap[2 * i] * L.amp_s[i], b = (float)kap[2 * i + 1] * L.amp_s[i];
    zr += cre * a - cim * b;
    zi += cre * b + cim * a;
    hh += (cre * cre + cim * cim) * (vv ? (float)vv[i] : L.amp_k[i]);
  }
  // with d_L marginalised the template is at 1 Mpc: zr, zi, hh are Z1, H1
  if (L.dist_marg) return distance_marg_logl(L, (double)zr, (double)zi, (double)hh);
  const float core = (L.phase_marg ? log_i0_f32(sqrtf(zr * zr + zi * zi)) : zr) - 0.5f * hh;
  return (double)core - 0.5 * L.DD;
}

// ---------------------------------------------------------------------------
// Chain control.
// ---------------------------------------------------------------------------
__device__ inline void finish_step(const SamplerConst& S, ChainState& ch, NSGlobal* g) {
  ch.phase = PH_NEW;
  if (++ch.step >= S.steps_per_dim * S.block_size[ch.block]) {
    ch.step = 0;
    if (++ch.block >= S.n_blocks) {
      ch.block = 0;
      if (++ch.sweep >= S.sweeps) {
        ch.done = 1;
        atomicAdd(&g->chains_done, 1);
      }
    }
  }
}

// Outcome of evaluating the proposal y with log-likelihood ly.  Returns true
// when the shrinkage phase accepts y (the caller moves the chain there and
// then calls finish_step); stepping-out and rejections are handled here.
__device__ inline bool apply_result(const SamplerConst& S, ChainState& ch, double ly, double logl_star,
                                    NSGlobal* g) {
  const bool ok = ly > logl_star;
  switch (ch.phase) {
    case PH_LEFT:
      if (ok) {
        ch.lo -= 1.0;
        if (++ch.n_out >= kMaxStepOut) {
          ch.phase = PH_RIGHT;
          ch.n_out = 0;
        }
      } else {
        ch.phase = PH_RIGHT;
        ch.n_out = 0;
      }
      return false;
    case PH_RIGHT:
      if (ok) {
        ch.hi += 1.0;
        if (++ch.n_out >= kMaxStepOut) {
          ch.phase = PH_SHRINK;
          ch.n_shrink = 0;
        }
      } else {
        ch.phase = PH_SHRINK;
        ch.n_shrink = 0;
      }
      return false;
    default:  // PH_SHRINK
      if (ok) return true;
      if (ch.t < 0.0)
        ch.lo = ch.t;
      else
        ch.hi = ch.t;
      if (++ch.n_shrink >= kMaxShrink) {
        ++ch.n_caps;
        finish_step(S, ch, g);
      }
      return false;
  }
}

__device__ inline void move_to_proposal(const SamplerConst& S, ChainState& ch, double ly) {
  for (int j = 0; j < S.ndim; ++j) ch.x[j] = ch.y[j];
  for (int j = 0; j < SWIG_N_PARAMS; ++j) ch.th[j] = ch.th_y[j];
  ch.lx = ly;
}

// New slice step: direction from the live covariance (n = L_b z, Sec. 2.3),
// or, with probability learn_mix, the learned direction exp(s_b) u_b / |u_b|
// of a live point drawn uniformly from the frozen snapshot; then a bracket
// [-r, 1 - r] of unit width at a uniform offset.
__device__ inline void start_step(const SamplerConst& S, ChainState& ch, const float* chol, const float* learn_out,
                                  int c, long long it) {
  const int b = ch.block, nb = S.block_size[b];
  for (int j = 0; j < S.ndim; ++j) ch.dir[j] = 0.0;
  bool learned = false;
  if (S.learn_on && learn_out && chain_uniform(S, ch, c, it) < (double)S.learn_mix) {
    const int row = min((int)(chain_uniform(S, ch, c, it) * (double)S.nlive), S.nlive - 1);
    const float* o = learn_out + (size_t)row * 32;
    float nrm2 = 0.0f;
    for (int r = 0; r < nb; ++r) {
      const float u = o[S.block_dims[b][r]];
      nrm2 = fmaf(u, u, nrm2);
    }
    const float inv = rsqrtf(nrm2 + 1e-12f);
    for (int r = 0; r < nb; ++r) {
      const int j = S.block_dims[b][r];
      const float s = fminf(fmaxf(o[13 + j], -30.0f), 5.0f);
      ch.dir[j] = (double)(expf(s) * o[j] * inv);
    }
    learned = true;
  }
  if (!learned) {
    float z[kMaxDim];
    for (int j = 0; j < nb; ++j) z[j] = chain_normal(S, ch, c, it);
    const float* Lb = chol + (size_t)b * kMaxDim * kMaxDim;
    for (int r = 0; r < nb; ++r) {
      float v = 0.0f;
      for (int q = 0; q <= r; ++q) v = fmaf(__ldcg(&Lb[r * kMaxDim + q]), z[q], v);
      ch.dir[S.block_dims[b][r]] = (double)v;
    }
  }
  const double r0 = chain_uniform(S, ch, c, it);
  ch.lo = -r0;
  ch.hi = 1.0 - r0;
  ch.phase = PH_LEFT;
  ch.n_out = 0;
  ch.n_shrink = 0;
}

// Advance chain c through the proposals that need no grid pass (outside the
// unit cube, or projection-only blocks, at most kFreeBudget of the latter per
// round) and leave the first full-likelihood proposal pending with its setup
// record in *rec.  Only the Gibbs block's slots are transformed and only the
// pieces of the record that the block moves are recomputed.  Lane 0 only.
template <bool MIXED>
__device__ __noinline__ void chain_advance_local(const LikeConst& L, const SamplerConst& S, const SamplerPtrs& P, int c,
                                    const double* kap_in, const double* vv_in, double ly_in, ChainState& ch,
                                    EvalRecord& rx, bool& rx_dirty, EvalRecord& rec, bool& rec_set,
                                    int& setup_fl) {
  NSGlobal* g = P.g;
  // written by CTA 0 at the boundary: read through L2, never a stale L1 line
  const double logl_star = __ldcg(&g->logl_star);
  const long long it = __ldcg(&g->iter);
  if (ch.done) return;
  const bool prof = (c == 0);
  long long tk = clock64();
  unsigned long long acc_res = 0, acc_step = 0, acc_prop = 0, acc_free = 0, acc_setup = 0, cnt_free = 0, cnt_setup = 0,
                     cnt_step = 0;
  struct Flush {
    NSGlobal* g;
    bool on;
    unsigned long long *a0, *a1, *a2, *a3, *a4, *n0, *n1, *n2;
    __device__ ~Flush() {
      if (!on) return;
      g->c_result += *a0;
      g->c_step += *a1;
      g->c_prop += *a2;
      g->c_free += *a3;
      g->c_setup += *a4;
      g->n_free += *n0;
      g->n_setup += *n1;
      g->n_step += *n2;
    }
  } flush{g, prof, &acc_res, &acc_step, &acc_prop, &acc_free, &acc_setup, &cnt_free, &cnt_setup, &cnt_step};
  if (ch.pending) {
    ch.pending = 0;
    ++ch.n_full;
    ++ch.n_evals;
    if (apply_result(S, ch, ly_in, logl_star, g)) {
      move_to_proposal(S, ch, ly_in);
      for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) ch.kap[j] = kap_in[j];
      if (vv_in)
        for (int i = 0; i < SWIG_MAX_DET; ++i) ch.vv[i] = vv_in[i];
      rx = rec;
      rx_dirty = true;
      ch.proj_dirty = 0;
      finish_step(S, ch, g);
    }
  }
  if (prof) {
    const long long t2 = clock64();
    acc_res += t2 - tk;
    tk = t2;
  }
  int free_left = kFreeBudget;
  for (int guard = 0; guard < 1 << 20 && !ch.done; ++guard) {
    const int b = ch.block;
    if (S.block_free[b] && free_left <= 0) return;  // resume next round
    if (ch.phase == PH_NEW) {
      start_step(S, ch, P.chol, P.learn_out, c, it);
      if (prof) {
        const long long t2 = clock64();
        acc_step += t2 - tk;
        cnt_step += 1;
        tk = t2;
      }
    }
    double t;
    if (ch.phase == PH_LEFT)
      t = ch.lo;
    else if (ch.phase == PH_RIGHT)
      t = ch.hi;
    else
      t = ch.lo + (ch.hi - ch.lo) * chain_uniform(S, ch, c, it);
    ch.t = t;
    const int nb = S.block_size[b];
    bool inside = true;
    for (int r = 0; r < nb; ++r) {
      const int j = S.block_dims[b][r];
      const double v = ch.x[j] + t * ch.dir[j];
      ch.y[j] = v;
      inside = inside && (v >= 0.0) && (v <= 1.0);
    }
    if (!inside) {
      apply_result(S, ch, -INFINITY, logl_star, g);
      continue;
    }
    for (int j = 0; j < S.ndim; ++j)
      if (ch.dir[j] == 0.0) ch.y[j] = ch.x[j];
    for (int q = 0; q < SWIG_N_PARAMS; ++q) ch.th_y[q] = ch.th[q];
    bool sky_block = false;
    for (int r = 0; r < nb; ++r) {
      const int j = S.block_dims[b][r], slot = S.slot_of_dim[j];
      // the sky angles go through FP64: the delays need them to ~1e-10
      ch.th_y[slot] = (MIXED && !(S.sky.on && (slot == 9 || slot == 10)))
                          ? prior_slot_inverse_f32(S.prior[slot], ch.y[j])
                          : prior_slot_inverse(S.prior[slot], ch.y[j]);
      sky_block = sky_block || slot == 9 || slot == 10;
    }
    if (S.sky.on && sky_block) sky_frame_to_radec(S.sky, ch.th_y[9], ch.th_y[10], &ch.th_y[9], &ch.th_y[10]);
    if (prof) {
      const long long t2 = clock64();
      acc_prop += t2 - tk;
      tk = t2;
    }
    if (S.block_free[b]) {
      --free_left;
      ++ch.n_evals;
      if (MIXED) {
        const double ly = free_loglike_mixed(L, ch.th_y, ch.kap, S.het ? ch.vv : nullptr);
        if (apply_result(S, ch, ly, logl_star, g)) {
          move_to_proposal(S, ch, ly);
          ch.proj_dirty = 1;
          finish_step(S, ch, g);
        }
        if (prof) {
          const long long t2 = clock64();
          acc_free += t2 - tk;
          cnt_free += 1;
          tk = t2;
        }
      } else {
        EvalRecord tmp = rx;
        tmp.valid = theta_valid(ch.th_y) ? 1 : 0;
        setup_amp(ch.th_y, &tmp);
        setup_projection(L, ch.th_y, &tmp);
        setup_combine(L, &tmp);
        double kre[SWIG_MAX_DET], kim[SWIG_MAX_DET];
        for (int i = 0; i < SWIG_MAX_DET; ++i) {
          kre[i] = ch.kap[2 * i];
          kim[i] = ch.kap[2 * i + 1];
        }
        const double ly = loglike_epilogue(L, tmp, kre, kim);
        if (apply_result(S, ch, ly, logl_star, g)) {
          move_to_proposal(S, ch, ly);
          rx = tmp;
          rx_dirty = true;
          finish_step(S, ch, g);
        }
      }
      continue;
    }
    rec = rx;
    setup_fl = S.block_flags[b] | (ch.proj_dirty ? (BF_AMP | BF_PROJ) : 0);
    rec.valid = theta_valid(ch.th_y) ? 1 : 0;
    rec_set = true;
    ch.pending = 1;
    P.pending[c] = 1;
    if (prof) {
      acc_setup += clock64() - tk;
      cnt_setup += 1;
    }
    return;
  }
}

// Chain control on local copies of the chain state and records (local
// memory is cached in L1; the global copies are read and written once).
// Lane 0 only.  Returns the set-up flags of the new pending proposal (its
// record in *rec_out still holds the current point's values for the pieces
// the block moves), or -1 when nothing is pending.
template <bool MIXED>
__device__ __noinline__ int chain_advance(const LikeConst& L, const SamplerConst& S, const SamplerPtrs& P, int c,
                                          const double* kap_in, double ly_in, EvalRecord* rec_out,
                                          const double* vv_in = nullptr) {
  if (P.chains[c].done) return -1;
  ChainState ch = P.chains[c];
  EvalRecord rx = P.recx[c];
  EvalRecord rec;
  if (ch.pending) rec = *rec_out;
  bool rx_dirty = false, rec_set = false;
  int fl = -1;
  chain_advance_local<MIXED>(L, S, P, c, kap_in, vv_in, ly_in, ch, rx, rx_dirty, rec, rec_set, fl);
  P.chains[c] = ch;
  if (rx_dirty) P.recx[c] = rx;
  if (rec_set) *rec_out = rec;
  return fl;
}

// The set-up of a pending proposal's record, one piece per lane: lane 0 the
// waveform coefficients (all, or only spin / tidal ones), lane 1 the
// amplitude, lanes 2.. the projection of each detector, lanes 8.. the time
// shift of each detector; then one lane per coefficient splits it into a
// double-float and one lane per detector forms C_i (lane 0 adds <h|h> in
// detector order).  All 32 lanes call it with the same fl (>= 0) and th (the
// proposal's theta).
__device__ __noinline__ void setup_record_warp(const LikeConst& L, const double* th, int fl, bool f32,
                                               EvalRecord* rec, int lane) {
  const bool valid = rec->valid != 0;
  // a sky move: the two FP64 sines/cosines of the delays on lanes 0 and 1 at
  // once (one call's latency), shared with the delay lanes
  double sl = 0.0, cl = 0.0, sd = 0.0, cd = 0.0;
  if (valid && (fl & BF_SKY)) {  // warp-uniform
    double sv, cv;
    sincos((lane & 1) ? th[10] : th[9] - L.gmst, &sv, &cv);
    sl = __shfl_sync(0xffffffffu, sv, 0);
    cl = __shfl_sync(0xffffffffu, cv, 0);
    sd = __shfl_sync(0xffffffffu, sv, 1);
    cd = __shfl_sync(0xffffffffu, cv, 1);
  }
  if (valid) {
    if (lane == 0) {
      if (fl & BF_INTR)
        setup_intrinsic(th, rec, false);
      else if (fl & (BF_SPIN | BF_TIDE))
        setup_intrinsic_partial(th, rec, (fl & BF_SPIN) != 0, (fl & BF_TIDE) != 0, false);
    } else if (lane == 1) {
      if (fl & BF_AMP) {
        if (f32)
          setup_amp_f32(th, rec);
        else
          setup_amp(th, rec);
      }
    } else if (lane >= 2 && lane < 2 + L.n_det) {
      if (fl & BF_PROJ) setup_projection_det(L, th, lane - 2, f32, rec);
    } else if (lane >= 8 && lane < 8 + L.n_det) {
      if (fl & BF_SKY)
        setup_delay_det_sc(L, th, lane - 8, sl, cl, sd, cd, rec);
      else if (fl & BF_TAU)
        setup_tc_det(th, lane - 8, rec);
    }
  } else if (lane == 0) {
    // invalid proposal: the record only has to say so (logL = -inf)
    rec->amp = 0.0;
  }
  __syncwarp();
  if (valid && (fl & (BF_INTR | BF_SPIN | BF_TIDE)) && lane < NBASIS) {
    const dfl v = df_from_double(rec->c[lane]);
    rec->c_hi[lane] = v.hi;
    rec->c_lo[lane] = v.lo;
  }
  double term = 0.0;
  if (lane < SWIG_MAX_DET) {
    const double cre = rec->amp * rec->pre[lane], cim = rec->amp * rec->pim[lane];
    rec->cre[lane] = cre;
    rec->cim[lane] = cim;
    if (lane < L.n_det) term = (cre * cre + cim * cim) * L.K[lane];
  }
  double hh = 0.0;
#pragma unroll
  for (int i = 0; i < SWIG_MAX_DET; ++i) hh += __shfl_sync(0xffffffffu, term, i);
  if (lane == 0) rec->hh = hh;
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Iteration boundary on CTA 0.
// ---------------------------------------------------------------------------
__device__ void block_reduce_max_sum(double* vals, int n, double* out_max, double* out_sumexp, double* s_tmp) {
  // two passes over vals[0..n): max, then sum exp(v - max); s_tmp holds at
  // least the block size rounded up to a power of two (tree over it, the
  // padding holding the operation's identity)
  const int nt = blockDim.x, tid = threadIdx.x;
  int np2 = 1;
  while (np2 < nt) np2 <<= 1;
  double m = -INFINITY;
  for (int i = tid; i < n; i += nt) m = fmax(m, vals[i]);
  s_tmp[tid] = m;
  if (tid + nt < np2) s_tmp[tid + nt] = -INFINITY;
  __syncthreads();
  for (int s = np2 / 2; s > 0; s >>= 1) {
    if (tid < s) s_tmp[tid] = fmax(s_tmp[tid], s_tmp[tid + s]);
    __syncthreads();
  }
  m = s_tmp[0];
  __syncthreads();
  double acc = 0.0;
  if (isfinite(m))
    for (int i = tid; i < n; i += nt) acc += exp(vals[i] - m);
  s_tmp[tid] = acc;
  if (tid + nt < np2) s_tmp[tid + nt] = 0.0;
  __syncthreads();
  for (int s = np2 / 2; s > 0; s >>= 1) {
    if (tid < s) s_tmp[tid] += s_tmp[tid + s];
    __syncthreads();
  }
  *out_max = m;
  *out_sumexp = s_tmp[0];
  __syncthreads();
}

// First half of the boundary: write the finished chains back into the live
// set and apply the launch's iteration limit and the termination rule.  Fills
// the sort keys in `smem` for the second half.  Returns false (status set)
// when the run stops here.
__device__ __noinline__ bool ns_boundary_check(const LikeConst& L, const SamplerConst& S, const SamplerPtrs& P,
                                               unsigned char* smem) {
  NSGlobal* g = P.g;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int m = S.nlive, k = S.nrep, d = S.ndim;
  if (g->need_writeback) {
    for (int c = tid; c < k; c += nt) {
      const ChainState& ch = P.chains[c];
      const int slot = __ldcg(&ch.slot);
      for (int j = 0; j < d; ++j) P.live_u[(size_t)slot * d + j] = __ldcg(&ch.x[j]);
      P.live_logl[slot] = __ldcg(&ch.lx);
      for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) P.live_kap[(size_t)slot * 2 * SWIG_MAX_DET + j] = __ldcg(&ch.kap[j]);
      for (int i = 0; i < SWIG_MAX_DET; ++i) P.live_vv[(size_t)slot * SWIG_MAX_DET + i] = __ldcg(&ch.vv[i]);
    }
    __syncthreads();
    if (tid == 0) g->need_writeback = 0;
  }
  __syncthreads();
  if (g->iters_launch >= S.max_iters) {
    if (tid == 0) g->status = ST_LIMIT;
    return false;
  }
  double* key = reinterpret_cast<double*>(smem);
  int* idx = reinterpret_cast<int*>(key + S.m_pow2);
  double* tmp = reinterpret_cast<double*>(idx + S.m_pow2);  // (nt rounded up to a power of two) doubles
  for (int i = tid; i < S.m_pow2; i += nt) {
    key[i] = i < m ? P.live_logl[i] : INFINITY;
    idx[i] = i;
  }
  __syncthreads();
  // termination: log Z_live = log X + log mean L_live
  double mx, se;
  block_reduce_max_sum(key, m, &mx, &se, tmp);
  const double logz_live = g->logx + mx + log(se / (double)m);
  const double logz = g->logz;
  if (isfinite(logz) && logz_live - logz < S.dlogz) {
    if (tid == 0) g->status = ST_TERMINATED;
    return false;
  }
  return true;
}

// Second half: sort, retire the k worst points, update log X / log Z and
// logL*, estimate the block Cholesky factors, start k chains at survivors.
__device__ __noinline__ void ns_boundary_advance(const LikeConst& L, const SamplerConst& S, const SamplerPtrs& P,
                                                 unsigned char* smem) {
  NSGlobal* g = P.g;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int m = S.nlive, k = S.nrep, d = S.ndim;
  double* key = reinterpret_cast<double*>(smem);
  int* idx = reinterpret_cast<int*>(key + S.m_pow2);
  double* tmp = reinterpret_cast<double*>(idx + S.m_pow2);
  // bitonic sort (ascending) of (logL, index)
  for (int kk = 2; kk <= S.m_pow2; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < S.m_pow2; i += nt) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool asc = (i & kk) == 0;
          const double a = key[i], b = key[ixj];
          if ((a > b) == asc || (a == b && ((idx[i] > idx[ixj]) == asc))) {
            key[i] = b;
            key[ixj] = a;
            const int t = idx[i];
            idx[i] = idx[ixj];
            idx[ixj] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  // deaths: w_j = L_j (X_{j-1} - X_j), log X_j = log X_0 - sum_{i<=j} 1/(m - i)
  const int base = g->n_dead;
  int np2 = 1;  // the reduction scratch spans the block size rounded up to a power of two
  while (np2 < nt) np2 <<= 1;
  double* logw = tmp + np2;  // k doubles
  for (int j = tid; j < k; j += nt) {
    const int s = idx[j];
    const double lwj = key[j] + (g->logx - P.harm[j]) + P.lw[m - j];
    logw[j] = lwj;
    P.dead_logl[base + j] = key[j];
    P.dead_logw[base + j] = lwj;
    for (int q = 0; q < d; ++q) P.dead_u[(size_t)(base + j) * d + q] = P.live_u[(size_t)s * d + q];
  }
  __syncthreads();
  double wm, ws;
  block_reduce_max_sum(logw, k, &wm, &ws, tmp);
  if (tid == 0) {
    const double a = g->logz, b = wm + log(ws);
    const double hi = fmax(a, b);
    g->logz = isfinite(hi) ? hi + log(exp(a - hi) + exp(b - hi)) : hi;
    g->logx -= P.harm[k];
    g->logl_star = key[k];
    g->n_dead = base + k;
  }
  // covariance of the live points (FP32; only a proposal scale) and block Cholesky
  float* mean = reinterpret_cast<float*>(logw + k);
  float* cov = mean + kMaxDim;  // kMaxDim x kMaxDim
  if (tid < d) {
    float acc = 0.0f;
    for (int i = 0; i < m; ++i) acc += (float)P.live_u[(size_t)i * d + tid];
    mean[tid] = acc / (float)m;
  }
  __syncthreads();
  if (tid < d * d) {
    const int a = tid / d, b = tid % d;
    if (b <= a) {
      float acc0 = 0.0f, acc1 = 0.0f;
      const float ma = mean[a], mb = mean[b];
      int i = 0;
      for (; i + 1 < m; i += 2) {
        acc0 = fmaf((float)P.live_u[(size_t)i * d + a] - ma, (float)P.live_u[(size_t)i * d + b] - mb, acc0);
        acc1 = fmaf((float)P.live_u[(size_t)(i + 1) * d + a] - ma, (float)P.live_u[(size_t)(i + 1) * d + b] - mb, acc1);
      }
      if (i < m) acc0 = fmaf((float)P.live_u[(size_t)i * d + a] - ma, (float)P.live_u[(size_t)i * d + b] - mb, acc0);
      const float v = (acc0 + acc1) / (float)(m - 1);
      cov[a * kMaxDim + b] = v;
      cov[b * kMaxDim + a] = v;
    }
  }
  __syncthreads();
  if (tid < S.n_blocks) {
    const int b = tid, nb = S.block_size[b];
    float* Lb = P.chol + (size_t)b * kMaxDim * kMaxDim;
    float tr = 0.0f;
    for (int r = 0; r < nb; ++r) tr += cov[S.block_dims[b][r] * kMaxDim + S.block_dims[b][r]];
    const float jitter = fmaxf(1e-6f * tr / (float)nb, 1e-30f);
    for (int r = 0; r < nb; ++r) {
      for (int q = 0; q <= r; ++q) {
        float s = cov[S.block_dims[b][r] * kMaxDim + S.block_dims[b][q]] + (r == q ? jitter : 0.0f);
        for (int p = 0; p < q; ++p) s -= Lb[r * kMaxDim + p] * Lb[q * kMaxDim + p];
        if (r == q)
          Lb[r * kMaxDim + r] = sqrtf(fmaxf(s, jitter));
        else
          Lb[r * kMaxDim + q] = s / Lb[q * kMaxDim + q];
      }
    }
  }
  __syncthreads();
  // chains: replace the c-th worst, start at a uniformly drawn survivor
  const long long it = g->iter;
  for (int c = tid; c < k; c += nt) {
    ChainState& ch = P.chains[c];
    const uint4 r = philox4x32_10(make_uint4(0u, (unsigned)c, (unsigned)it, 1u), S.key0, S.key1);
    int pick = (int)(u01_from(r) * (double)(m - k));
    pick = min(pick, m - k - 1);
    const int s = idx[k + pick];
    ch.slot = idx[c];
    for (int j = 0; j < d; ++j) ch.x[j] = P.live_u[(size_t)s * d + j];
    ch.lx = P.live_logl[s];
    for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) ch.kap[j] = P.live_kap[(size_t)s * 2 * SWIG_MAX_DET + j];
    for (int i = 0; i < SWIG_MAX_DET; ++i) ch.vv[i] = P.live_vv[(size_t)s * SWIG_MAX_DET + i];
    prior_map(S.prior, ch.x, ch.th, &S.sky);
    setup_record(L, ch.th, &P.recx[c]);
    ch.proj_dirty = 0;
    ch.block = ch.step = ch.sweep = 0;
    ch.phase = PH_NEW;
    ch.pending = 0;
    ch.done = 0;
    ch.ctr = 0;
    ch.side = 0;
    ch.n_out_r = 0;
    P.pending[c] = 0;
    P.req[c] = 0;
    P.done_cnt[c] = 0;
    if (S.par_out) {
      P.req[k + c] = 0;
      P.done_cnt[k + c] = 0;
    }
  }
  __syncthreads();
  if (tid == 0) {
    g->chains_done = 0;
    g->iter = it + 1;
    g->iters_launch += 1;
    g->need_writeback = 1;
  }
}

__device__ void ns_boundary(const LikeConst& L, const SamplerConst& S, const SamplerPtrs& P, unsigned char* smem) {
  if (ns_boundary_check(L, S, P, smem)) ns_boundary_advance(L, S, P, smem);
}

// ---------------------------------------------------------------------------
// The persistent kernel, dataflow form.  Within an NS iteration nothing
// waits on a grid-wide barrier: warp 0 of each CTA runs the control of the
// chains homed there, and publishes each full-likelihood request by bumping
// the chain's sequence number after writing its record; warps 1.. of every
// CTA claim (chain, request) pairs as they appear and evaluate the CTA's
// slice of the grid for them (one warp per pair), then count themselves in
// done_cnt.  A chain's control resumes once all CTAs have counted.  The
// per-slice sums are written in a fixed place and added over slices in a
// fixed order, so results do not depend on timing.  Every wait is bounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Copy the part of a record that a sweep unit reads (the double-float phase
// coefficients and the time shifts: one contiguous run of words), written by
// another SM, into shared memory (through L2).
static_assert(offsetof(EvalRecord, c_lo) > offsetof(EvalRecord, c_hi) &&
                  offsetof(EvalRecord, tau) > offsetof(EvalRecord, c_lo) &&
                  offsetof(EvalRecord, tau_hi) > offsetof(EvalRecord, tau) &&
                  offsetof(EvalRecord, tau_lo) > offsetof(EvalRecord, tau_hi),
              "the sweep's fields of EvalRecord are one run");
// The FP64 sweep (MIXED false) also reads the FP64 coefficients c, which
// precede that run.
template <bool MIXED = true>
__device__ __forceinline__ void load_record_cg(const EvalRecord* src, EvalRecord* dst, int lane) {
  static_assert(offsetof(EvalRecord, c) == 0 && offsetof(EvalRecord, c_hi) > 0, "c leads the record");
  constexpr int w0 = MIXED ? (int)(offsetof(EvalRecord, c_hi) / 4) : 0;
  constexpr int w1 = (int)((offsetof(EvalRecord, tau_lo) + sizeof(float) * SWIG_MAX_DET) / 4);
  const unsigned* s = reinterpret_cast<const unsigned*>(src);
  unsigned* d = reinterpret_cast<unsigned*>(dst);
  for (int w = w0 + lane; w < w1; w += 32) d[w] = __ldcg(s + w);
  __syncwarp();
}

// done_cnt += v with release semantics (orders the unit's partial writes,
// made visible to lane 0 by the preceding __syncwarp, before the count).
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One control step of chain c by a whole warp: add the slice partials of the
// finished request (fixed order), advance the chain's slice state machine and,
// when it needs a full likelihood, set up its record and publish the request.
// Returns true while the chain needs another control step right away
// (projection-only budget used up), false once it waits for a request or is
// done.
template <int NDET, bool MIXED>
__device__ bool flow_control(const LikeConst& L, const SamplerConst& S, const DeviceBuffers& B, const SamplerPtrs& P,
                             int c, int lane) {
  NSGlobal* g = P.g;
  double kap_y[2 * SWIG_MAX_DET];
#pragma unroll
  for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) kap_y[j] = 0.0;
  double ly = 0.0;
  const bool pend = P.chains[c].pending != 0;
  if (pend) {
    double acc[2 * SWIG_MAX_DET];
#pragma unroll
    for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) acc[j] = 0.0;
    const int n_units = L.n_slices * S.flow_parts;
    for (int s2 = lane; s2 < n_units; s2 += 32) {
#pragma unroll
      for (int j = 0; j < 2 * NDET; ++j)
        acc[j] += MIXED ? (double)__ldcg(&B.partials32[((size_t)c * n_units + s2) * kPartialStride + j])
                        : __ldcg(&B.partials64[((size_t)c * n_units + s2) * kPartialStride + j]);
    }
#pragma unroll
    for (int j = 0; j < 2 * NDET; ++j)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
#pragma unroll
    for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) kap_y[j] = acc[j];
    if (lane == 0) {
      double kre[SWIG_MAX_DET], kim[SWIG_MAX_DET];
      for (int i = 0; i < SWIG_MAX_DET; ++i) {
        kre[i] = kap_y[2 * i];
        kim[i] = kap_y[2 * i + 1];
      }
      ly = loglike_epilogue(L, B.rec[c], kre, kim);
    }
  }
  int fl = -1, done = 0;
  if (lane == 0) {
    if (pend) P.pending[c] = 0;
    fl = chain_advance<MIXED>(L, S, P, c, kap_y, ly, &B.rec[c]);
    done = P.chains[c].done;
  }
  fl = __shfl_sync(0xffffffffu, fl, 0);
  done = __shfl_sync(0xffffffffu, done, 0);
  __syncwarp();
  if (fl >= 0) {
    const long long ts = clock64();
    setup_record_warp(L, P.chains[c].th_y, fl, MIXED, &B.rec[c], lane);
    if (lane == 0) {
      if (c == 0) g->c_setup += clock64() - ts;
      P.done_cnt[c] = 0;
      __threadfence();
      // sequence number and unit width in one word (one unit per slice)
      st_release(&P.req[c], (((P.req[c] >> 3) + 1) << 3) | S.flow_parts);
    }
    __syncwarp();
    return false;
  }
  return !done;
}


// ---------------------------------------------------------------------------
// Warp-parallel chain control (mixed-precision full-grid sampler).
//
// The control warp keeps the state of the chains homed on its CTA in shared
// memory for the whole NS iteration (copied in after the boundary and back
// before the next one).  During a control step the state lives in registers
// spread over the lanes: the scalars are uniform across the warp; lane j
// holds dimension j of x, y and the slice direction, slot j of theta and of
// the proposal's theta, and component j of the cached kappa sums.  The
// per-dimension work of a proposal (the point on the slice, the unit-cube
// test, the prior transform, the validity test) is one step across the
// lanes instead of a loop, the direction's normal draws and its Cholesky
// product run one row per lane, a projection-only evaluation runs one
// detector per lane, and records move between shared and global memory with
// the whole warp.  Each value is formed by the same operations as in
// chain_advance_local, and the Philox counters are drawn in the same order,
// so the random stream of a chain is unchanged.
// ---------------------------------------------------------------------------
constexpr unsigned kFull = 0xffffffffu;

struct WarpChain {
  double x, y, dir, th, thy, kap, vv;  // lane-indexed, see above (vv: detector i on lane i)
  double lx, lo, hi, t;
  int block, step, sweep, phase, n_out, n_shrink, done, proj_dirty, n_caps, side, n_out_r;
  unsigned ctr;
  long long n_evals, n_full;
};

__device__ __forceinline__ void wc_load(const ChainState& ch, WarpChain& w, int lane) {
  const int l = lane < kMaxDim ? lane : 0;
  w.x = ch.x[l];
  w.y = ch.y[l];
  w.dir = ch.dir[l];
  w.th = ch.th[l];
  w.thy = ch.th_y[l];
  w.kap = lane < 2 * SWIG_MAX_DET ? ch.kap[lane] : 0.0;
  w.vv = lane < SWIG_MAX_DET ? ch.vv[lane] : 0.0;
  w.lx = ch.lx;
  w.lo = ch.lo;
  w.hi = ch.hi;
  w.t = ch.t;
  w.block = ch.block;
  w.step = ch.step;
  w.sweep = ch.sweep;
  w.phase = ch.phase;
  w.n_out = ch.n_out;
  w.n_shrink = ch.n_shrink;
  w.done = ch.done;
  w.proj_dirty = ch.proj_dirty;
  w.n_caps = ch.n_caps;
  w.side = ch.side;
  w.n_out_r = ch.n_out_r;
  w.ctr = ch.ctr;
  w.n_evals = ch.n_evals;
  w.n_full = ch.n_full;
}

__device__ __forceinline__ void wc_store(ChainState& ch, const WarpChain& w, int lane) {
  if (lane < kMaxDim) {
    ch.x[lane] = w.x;
    ch.y[lane] = w.y;
    ch.dir[lane] = w.dir;
    ch.th[lane] = w.th;
    ch.th_y[lane] = w.thy;
  }
  if (lane < 2 * SWIG_MAX_DET) ch.kap[lane] = w.kap;
  if (lane < SWIG_MAX_DET) ch.vv[lane] = w.vv;
  if (lane == 0) {
    ch.lx = w.lx;
    ch.lo = w.lo;
    ch.hi = w.hi;
    ch.t = w.t;
    ch.block = w.block;
    ch.step = w.step;
    ch.sweep = w.sweep;
    ch.phase = w.phase;
    ch.n_out = w.n_out;
    ch.n_shrink = w.n_shrink;
    ch.done = w.done;
    ch.proj_dirty = w.proj_dirty;
    ch.n_caps = w.n_caps;
    ch.side = w.side;
    ch.n_out_r = w.n_out_r;
    ch.ctr = w.ctr;
    ch.n_evals = w.n_evals;
    ch.n_full = w.n_full;
  }
  __syncwarp();
}

// Copy n bytes (a multiple of 4) with the whole warp.
__device__ __forceinline__ void warp_copy(void* dst, const void* src, int n, int lane) {
  const unsigned* s4 = static_cast<const unsigned*>(src);
  unsigned* d4 = static_cast<unsigned*>(dst);
  for (int q = lane; q < n / 4; q += 32) d4[q] = s4[q];
  __syncwarp();
}

// The same from global memory written by another SM (through L2).
__device__ __forceinline__ void warp_copy_cg(void* dst, const void* src, int n, int lane) {
  const unsigned* s4 = static_cast<const unsigned*>(src);
  unsigned* d4 = static_cast<unsigned*>(dst);
  for (int q = lane; q < n / 4; q += 32) d4[q] = __ldcg(s4 + q);
  __syncwarp();
}

__device__ __forceinline__ double wc_uniform(const SamplerConst& S, WarpChain& w, int c, long long it) {
  return u01_from(philox4x32_10(make_uint4(w.ctr++, (unsigned)c, (unsigned)it, 0u), S.key0, S.key1));
}

__device__ __forceinline__ void wc_finish_step(const SamplerConst& S, WarpChain& w, NSGlobal* g, int lane) {
  w.phase = PH_NEW;
  if (++w.step >= S.steps_per_dim * S.block_size[w.block]) {
    w.step = 0;
    if (++w.block >= S.n_blocks) {
      w.block = 0;
      if (++w.sweep >= S.sweeps) {
        w.done = 1;
        if (lane == 0) atomicAdd(&g->chains_done, 1);
      }
    }
  }
}

// apply_result on the warp's copy (uniform).
__device__ __forceinline__ bool wc_apply(const SamplerConst& S, WarpChain& w, double ly, double logl_star, NSGlobal* g,
                                         int lane) {
  const bool ok = ly > logl_star;
  switch (w.phase) {
    case PH_LEFT:
      if (ok) {
        w.lo -= 1.0;
        if (++w.n_out >= kMaxStepOut) {
          w.phase = PH_RIGHT;
          w.n_out = 0;
        }
      } else {
        w.phase = PH_RIGHT;
        w.n_out = 0;
      }
      return false;
    case PH_RIGHT:
      if (ok) {
        w.hi += 1.0;
        if (++w.n_out >= kMaxStepOut) {
          w.phase = PH_SHRINK;
          w.n_shrink = 0;
        }
      } else {
        w.phase = PH_SHRINK;
        w.n_shrink = 0;
      }
      return false;
    default:  // PH_SHRINK
      if (ok) return true;
      if (w.t < 0.0)
        w.lo = w.t;
      else
        w.hi = w.t;
      if (++w.n_shrink >= kMaxShrink) {
        ++w.n_caps;
        wc_finish_step(S, w, g, lane);
      }
      return false;
  }
}

__device__ __forceinline__ bool wc_in_block(const SamplerConst& S, int b, int lane) {
  return lane < S.ndim && ((S.block_mask[b] >> lane) & 1u);
}

// start_step across the warp.
__device__ __forceinline__ void wc_start_step(const SamplerConst& S, WarpChain& w, const float* chol,
                                              const float* learn_out, int c, long long it, int lane) {
  const int b = w.block, nb = S.block_size[b];
  const bool inb = wc_in_block(S, b, lane);
  w.dir = 0.0;
  bool learned = false;
  if (S.learn_on && learn_out && wc_uniform(S, w, c, it) < (double)S.learn_mix) {
    const int row = min((int)(wc_uniform(S, w, c, it) * (double)S.nlive), S.nlive - 1);
    const float* o = learn_out + (size_t)row * 32;
    float nrm2 = 0.0f;
    for (int r = 0; r < nb; ++r) {
      const float u = o[S.block_dims[b][r]];
      nrm2 = fmaf(u, u, nrm2);
    }
    const float inv = rsqrtf(nrm2 + 1e-12f);
    if (inb) {
      const float sv = fminf(fmaxf(o[13 + lane], -30.0f), 5.0f);
      w.dir = (double)(expf(sv) * o[lane] * inv);
    }
    learned = true;
  }
  if (!learned) {
    // z_r, r < nb, one Philox block each at consecutive counters (chain_normal)
    float z = 0.0f;
    if (lane < nb) {
      const uint4 r = philox4x32_10(make_uint4(w.ctr + (unsigned)lane, (unsigned)c, (unsigned)it, 0u), S.key0, S.key1);
      const float u1 = ((float)(r.x >> 8) + 1.0f) * (1.0f / 16777216.0f);
      const float u2 = (float)(r.y >> 8) * (1.0f / 16777216.0f);
      z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    }
    w.ctr += (unsigned)nb;
    // lane r forms row r of L_b z
    const float* Lb = chol + (size_t)b * kMaxDim * kMaxDim;
    float v = 0.0f;
    for (int q = 0; q < nb; ++q) {
      const float zq = __shfl_sync(kFull, z, q);
      if (lane < nb && q <= lane) v = fmaf(__ldcg(&Lb[lane * kMaxDim + q]), zq, v);  // CTA 0 writes L_b
    }
    // ... and dimension j of the block takes row block_rank[j]
    const float vd = __shfl_sync(kFull, v, lane < S.ndim ? S.block_rank[lane] : 0);
    if (inb) w.dir = (double)vd;
  }
  const double r0 = wc_uniform(S, w, c, it);
  w.lo = -r0;
  w.hi = 1.0 - r0;
  // both ends at once where the evaluations are requests to the sweep (the
  // same evaluations and decisions as left, then right)
  w.phase = (S.par_out && !S.block_free[b]) ? PH_OUT : PH_LEFT;
  w.side = 3;
  w.n_out = 0;
  w.n_out_r = 0;
  w.n_shrink = 0;
}

// free_loglike_mixed across the warp: lane i < NDET forms detector i's terms
// (HET: <h|h>_i from the cached vv_i, else the constant K_i A1^2); lane 0 adds
// them in detector order and finishes.
template <int NDET, bool HET>
__device__ __forceinline__ double wc_free_loglike(const LikeConst& L, const WarpChain& w, int lane) {
  const float tf = (float)w.thy, kf = (float)w.kap;
  const float mc = __shfl_sync(kFull, tf, 0), dl = __shfl_sync(kFull, tf, 6);
  const float iota = __shfl_sync(kFull, tf, 7), psi = __shfl_sync(kFull, tf, 8);
  const float ra = __shfl_sync(kFull, tf, 9), dec = __shfl_sync(kFull, tf, 10), phic = __shfl_sync(kFull, tf, 12);
  const int di = lane < NDET ? lane : 0;
  const float ka = __shfl_sync(kFull, kf, 2 * di), kb = __shfl_sync(kFull, kf, 2 * di + 1);
  const float hk = HET ? (float)w.vv : L.amp_k[di];
  if (!(mc > 0.0f && dl > 0.0f)) return -INFINITY;
  float tr = 0.0f, ti = 0.0f, th = 0.0f;
  if (lane < NDET) {
    const float rel = exp2f(0.8333333333f * log2f(mc)) / dl;
    float sl, cl, sd, cd, sp, cp;
    sincosf(ra - (float)L.gmst, &sl, &cl);
    sincosf(dec, &sd, &cd);
    sincosf(psi, &sp, &cp);
    const float east[3] = {-sl, cl, 0.0f};
    const float north[3] = {-sd * cl, -sd * sl, cd};
    float X[3], Y[3];
    for (int k = 0; k < 3; ++k) {
      X[k] = -cp * east[k] + sp * north[k];
      Y[k] = sp * east[k] + cp * north[k];
    }
    const float ci = cosf(iota);
    const float plus = 0.5f * (1.0f + ci * ci), cross = -ci;
    float sph = 0.0f, cph = 1.0f;
    if (!L.phase_marg) sincosf(phic, &sph, &cph);
    float d[6];
    for (int q = 0; q < 6; ++q) d[q] = (float)L.dten[di][q];
    auto form = [&d](const float* a, const float* b) {
      return a[0] * (d[0] * b[0] + d[1] * b[1] + d[2] * b[2]) + a[1] * (d[1] * b[0] + d[3] * b[1] + d[4] * b[2]) +
             a[2] * (d[2] * b[0] + d[4] * b[1] + d[5] * b[2]);
    };
    const float fp = form(X, X) - form(Y, Y), fx = 2.0f * form(X, Y);
    const float re0 = rel * fp * plus, im0 = rel * fx * cross;
    const float cre = re0 * cph - im0 * sph, cim = re0 * sph + im0 * cph;
    const float a = ka * L.amp_s[di], b = kb * L.amp_s[di];
    tr = cre * a - cim * b;
    ti = cre * b + cim * a;
    th = (cre * cre + cim * cim) * hk;
  }
  float zr = 0.0f, zi = 0.0f, hh = 0.0f;
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
    zr += __shfl_sync(kFull, tr, i);
    zi += __shfl_sync(kFull, ti, i);
    hh += __shfl_sync(kFull, th, i);
  }
  double out = 0.0;
  if (lane == 0) {
    if (L.dist_marg) {
      out = distance_marg_logl(L, (double)zr, (double)zi, (double)hh);
    } else {
      const float core = (L.phase_marg ? log_i0_f32(sqrtf(zr * zr + zi * zi)) : zr) - 0.5f * hh;
      out = (double)core - 0.5 * L.DD;
    }
  }
  return __shfl_sync(kFull, out, 0);
}

// The result of chain c's finished request: the slice partials added in a
// fixed order as double-float sums on the FP32 pipe (each lane takes units
// lane, lane + 32, ..., error-free two-sums, then a butterfly of double-float
// adds; lane 0's totals are the result), each component rounded once to FP64
// on its own lane (kapc: lane j holds component j), and the FP64 epilogue of
// Eq. 2 with one detector's terms per lane (ly, on every lane).
template <int NDET>
__device__ __forceinline__ void wc_result(const LikeConst& L, const SamplerConst& S, const DeviceBuffers& B, int c,
                                          int lane, double& kapc, double& ly) {
  dfl acc[2 * NDET];
#pragma unroll
  for (int j = 0; j < 2 * NDET; ++j) acc[j] = dfl{0.0f, 0.0f};
  const int n_units = L.n_slices * S.flow_parts;
  for (int s0 = lane; s0 < n_units; s0 += 128) {
    // four units' loads in flight at once; a unit past the end adds zeros
    float v[4][2 * NDET];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s2 = s0 + 32 * q;
      const float* pp = &B.partials32[((size_t)c * n_units + min(s2, n_units - 1)) * kPartialStride];
#pragma unroll
      for (int j = 0; j < 2 * NDET; ++j) v[q][j] = s2 < n_units ? __ldcg(pp + j) : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int j = 0; j < 2 * NDET; ++j) {
        const dfl t = two_sum(acc[j].hi, v[q][j]);
        acc[j] = fast_two_sum(t.hi, __fadd_rn(t.lo, acc[j].lo));
      }
  }
#pragma unroll
  for (int j = 0; j < 2 * NDET; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const dfl b = {__shfl_xor_sync(kFull, acc[j].hi, o), __shfl_xor_sync(kFull, acc[j].lo, o)};
      acc[j] = df_add(acc[j], b);
    }
  float hi = 0.0f, lo = 0.0f;
#pragma unroll
  for (int j = 0; j < 2 * NDET; ++j) {
    const float h0 = __shfl_sync(kFull, acc[j].hi, 0), l0 = __shfl_sync(kFull, acc[j].lo, 0);
    if (lane == j) {
      hi = h0;
      lo = l0;
    }
  }
  kapc = lane < 2 * NDET ? (double)hi + (double)lo : 0.0;
  const EvalRecord& r = B.rec[c];
  // detector i's terms of Z = sum_i C_i kappa_i inv_scale_i on lane i
  const int di = lane < NDET ? lane : 0;
  const double kre = __shfl_sync(kFull, kapc, 2 * di), kim = __shfl_sync(kFull, kapc, 2 * di + 1);
  double tr = 0.0, ti = 0.0;
  if (lane < NDET) {
    const double a = kre * L.inv_scale[di], b = kim * L.inv_scale[di];
    tr = r.cre[di] * a - r.cim[di] * b;
    ti = r.cre[di] * b + r.cim[di] * a;
  }
  double zr = __shfl_sync(kFull, tr, 0), zi = __shfl_sync(kFull, ti, 0);
#pragma unroll
  for (int i = 1; i < NDET; ++i) {
    zr += __shfl_sync(kFull, tr, i);
    zi += __shfl_sync(kFull, ti, i);
  }
  double out = 0.0;
  if (lane == 0) {
    if (!r.valid) {
      out = -INFINITY;
    } else if (L.dist_marg) {
      out = distance_marg_logl(L, zr, zi, r.hh);
    } else {
      const double base = -0.5 * r.hh - 0.5 * L.DD;
      if (L.phase_marg) {
        const double x = sqrt(zr * zr + zi * zi);
        out = (L.fast_epilogue ? x + (double)log_i0e_f32((float)x) : log_bessel_i0(x)) + base;
      } else {
        out = zr + base;
      }
    }
  }
  ly = __shfl_sync(kFull, out, 0);
}

// One control step of chain c (state `ch` and current-point record `rx` in
// shared memory) by the whole warp: the result of its pending full
// evaluation, then the chain's slice steps up to the next full-likelihood
// proposal, whose record is set up in B.rec[c].  Full grid (HET false): the
// result is read from the slice partials and the proposal is published as a
// request to every CTA.  Heterodyned (HET true): the caller evaluates the
// proposal itself and passes the result back (het_ly on every lane,
// het_kap: component j on lane j, het_vv: detector i on lane i).  Returns
// CTL_WAIT (published, or the chain is done), CTL_AGAIN (projection-only
// budget used up: call again) or CTL_EVAL (HET: record set up, evaluate it).
enum { CTL_WAIT = 0, CTL_AGAIN = 1, CTL_EVAL = 2 };

// The proposal at bracket coordinate t of block b: the point y = x + t n on
// the block's dimensions (lane j: dimension j) and its theta (lane s: slot s).
// Returns false (and leaves theta alone) when y leaves the unit cube.
__device__ __forceinline__ bool wc_proposal(const SamplerConst& S, WarpChain& w, int b, double t, int lane) {
  const bool inb = wc_in_block(S, b, lane);
  if (lane < S.ndim) w.y = inb ? w.x + t * w.dir : w.x;
  const bool inside = __all_sync(kFull, !inb || (w.y >= 0.0 && w.y <= 1.0));
  if (!inside) return false;
  double v = 0.0;
  if (inb) {
    const int slot = S.slot_of_dim[lane];
    // the sky angles go through FP64: the delays need them to ~1e-10
    v = (S.sky.on && (slot == 9 || slot == 10)) ? prior_slot_inverse(S.prior[slot], w.y)
                                                : prior_slot_inverse_f32(S.prior[slot], w.y);
  }
  const int src = lane < SWIG_N_PARAMS ? S.dim_of_slot[lane] : -1;
  const double vs = __shfl_sync(kFull, v, src >= 0 ? src : 0);
  w.thy = (src >= 0 && ((S.block_mask[b] >> src) & 1u)) ? vs : w.th;
  if (S.sky.on && (S.block_flags[b] & BF_SKY)) {
    const double az = __shfl_sync(kFull, w.thy, 9), zen = __shfl_sync(kFull, w.thy, 10);
    double ra = 0.0, dec = 0.0;
    if (lane == 0) sky_frame_to_radec(S.sky, az, zen, &ra, &dec);
    ra = __shfl_sync(kFull, ra, 0);
    dec = __shfl_sync(kFull, dec, 0);
    if (lane == 9) w.thy = ra;
    if (lane == 10) w.thy = dec;
  }
  return true;
}

// Set up the record of the proposal in w.thy in request slot `slot` (the
// current point's record with block b's pieces recomputed) and, unless the
// caller evaluates it itself (HET), publish it to every CTA.
template <bool HET>
__device__ __forceinline__ void wc_publish(const LikeConst& L, const SamplerConst& S, const DeviceBuffers& B,
                                           const SamplerPtrs& P, int slot, int b, ChainState& ch,
                                           const EvalRecord& rx, const WarpChain& w, int lane) {
  const int fl = S.block_flags[b] | (w.proj_dirty ? (BF_AMP | BF_PROJ) : 0);
  const bool fin = lane >= SWIG_N_PARAMS || isfinite(w.thy);
  const double t0v = __shfl_sync(kFull, w.thy, 0), t1v = __shfl_sync(kFull, w.thy, 1);
  const double t6v = __shfl_sync(kFull, w.thy, 6);
  const bool valid = __all_sync(kFull, fin) && t0v > 0.0 && t1v > 0.0 && t1v <= 1.0 && t6v > 0.0;
  if (lane < SWIG_N_PARAMS) ch.th_y[lane] = w.thy;
  warp_copy(&B.rec[slot], &rx, sizeof(EvalRecord), lane);
  if (lane == 0) B.rec[slot].valid = valid ? 1 : 0;
  __syncwarp();
  setup_record_warp(L, ch.th_y, fl, true, &B.rec[slot], lane);
  if (!HET && lane == 0) {
    P.done_cnt[slot] = 0;
    __threadfence();
    // sequence number and unit width in one word
    st_release(&P.req[slot], (((P.req[slot] >> 3) + 1) << 3) | S.flow_parts);
  }
}

// One control step of chain c (state `ch` and current-point record `rx` in
// shared memory) by the whole warp: the results of its finished full
// evaluations, then the chain's slice steps up to the next full-likelihood
// proposal(s), whose records are set up in B.rec.  Full grid (HET false): a
// result is read from the slice partials and a proposal is published as a
// request to every CTA; with S.par_out the two ends of a bracket step out at
// once (left end in slot c, right end in slot nrep + c, ch.pending bits 0 and
// 1).  Heterodyned (HET true): the caller evaluates the proposal itself and
// passes the result back (het_ly on every lane, het_kap: component j on lane
// j, het_vv: detector i on lane i).  Returns CTL_WAIT (published, or the
// chain is done), CTL_AGAIN (projection-only budget used up: call again) or
// CTL_EVAL (HET: record set up, evaluate it).
template <int NDET, bool HET>
__device__ __forceinline__ int control_step_warp(const LikeConst& L, const SamplerConst& S, const DeviceBuffers& B,
                                 const SamplerPtrs& P, int c, ChainState& ch, EvalRecord& rx, int lane,
                                 double het_ly = 0.0, double het_kap = 0.0, double het_vv = 0.0) {
  NSGlobal* g = P.g;
  if (ch.done) return CTL_WAIT;
  const bool prof = (c == 0) && lane == 0;
  long long tk = clock64();
  unsigned long long acc_res = 0, acc_step = 0, acc_prop = 0, acc_free = 0, acc_setup = 0, cnt_free = 0,
                     cnt_setup = 0, cnt_step = 0;
  // written by CTA 0 at the boundary: read through L2, never a stale L1 line
  const double logl_star = __ldcg(&g->logl_star);
  const long long it = __ldcg(&g->iter);
  const int target = L.n_slices * S.flow_parts;
  WarpChain w;
  wc_load(ch, w, lane);
  int pend = ch.pending;
  // finished requests (one call site for the result, to keep the inlined
  // control small): an end of a two-ended step-out, or the chain's proposal
  for (int sd = 0; sd < 2; ++sd) {
    if (!((pend >> sd) & 1)) continue;
    const int slot = sd ? S.nrep + c : c;
    if (w.phase == PH_OUT) {
      int fin = 0;
      if (lane == 0) fin = ld_acquire(&P.done_cnt[slot]) >= target;
      if (!__shfl_sync(kFull, fin, 0)) continue;
    }
    double kapc = het_kap, ly = het_ly;
    if (!HET) wc_result<NDET>(L, S, B, slot, lane, kapc, ly);
    pend &= ~(1 << sd);
    ++w.n_full;
    ++w.n_evals;
    if (w.phase == PH_OUT) {  // extend this end while inside the slice
      const bool ok = ly > logl_star;
      if (sd == 0) {
        if (ok) w.lo -= 1.0;
        if (!ok || ++w.n_out >= kMaxStepOut) w.side &= ~1;
      } else {
        if (ok) w.hi += 1.0;
        if (!ok || ++w.n_out_r >= kMaxStepOut) w.side &= ~2;
      }
    } else if (wc_apply(S, w, ly, logl_star, g, lane)) {
      w.x = w.y;
      w.th = w.thy;
      w.lx = ly;
      w.kap = kapc;
      if (HET) w.vv = het_vv;
      warp_copy(&rx, &B.rec[c], sizeof(EvalRecord), lane);
      w.proj_dirty = 0;
      wc_finish_step(S, w, g, lane);
    }
  }
  if (prof) {
    const long long t2 = clock64();
    acc_res += t2 - tk;
    tk = t2;
  }
  int free_left = kFreeBudget;
  int status = CTL_WAIT;
  for (int guard = 0; guard < 1 << 20 && !w.done; ++guard) {
    const int b = w.block;
    int sd = 0;  // PH_OUT: the end to issue next (0 left, 1 right)
    if (w.phase == PH_OUT) {
      sd = ((w.side & 1) && !(pend & 1)) ? 0 : ((w.side & 2) && !(pend & 2)) ? 1 : -1;
      if (sd < 0) {
        if (pend) break;  // wait for the requests in flight
        w.phase = PH_SHRINK;  // both ends done
        w.n_shrink = 0;
        continue;
      }
    } else {
      if (S.block_free[b] && free_left <= 0) {  // resume next round
        status = CTL_AGAIN;
        break;
      }
      if (w.phase == PH_NEW) {
        wc_start_step(S, w, P.chol, P.learn_out, c, it, lane);
        if (prof) {
          const long long t2 = clock64();
          acc_step += t2 - tk;
          cnt_step += 1;
          tk = t2;
        }
        continue;
      }
    }
    double t;
    if (w.phase == PH_OUT)
      t = sd ? w.hi : w.lo;
    else if (w.phase == PH_LEFT)
      t = w.lo;
    else if (w.phase == PH_RIGHT)
      t = w.hi;
    else
      t = w.lo + (w.hi - w.lo) * wc_uniform(S, w, c, it);
    if (w.phase != PH_OUT) w.t = t;
    if (!wc_proposal(S, w, b, t, lane)) {  // outside the unit cube
      if (w.phase == PH_OUT)
        w.side &= ~(1 << sd);
      else
        wc_apply(S, w, -INFINITY, logl_star, g, lane);
      continue;
    }
    if (prof) {
      const long long t2 = clock64();
      acc_prop += t2 - tk;
      tk = t2;
    }
    if (w.phase != PH_OUT && S.block_free[b]) {
      --free_left;
      ++w.n_evals;
      const double ly = wc_free_loglike<NDET, HET>(L, w, lane);
      if (wc_apply(S, w, ly, logl_star, g, lane)) {
        w.x = w.y;
        w.th = w.thy;
        w.lx = ly;
        w.proj_dirty = 1;
        wc_finish_step(S, w, g, lane);
      }
      if (prof) {
        const long long t2 = clock64();
        acc_free += t2 - tk;
        cnt_free += 1;
        tk = t2;
      }
      continue;
    }
    // a full evaluation: published as a request (slot c, or nrep + c for the
    // right end of a two-ended step-out)
    wc_publish<HET>(L, S, B, P, sd == 1 ? S.nrep + c : c, b, ch, rx, w, lane);
    pend |= sd == 1 ? 2 : 1;
    if (prof) {
      acc_setup += clock64() - tk;
      cnt_setup += 1;
      tk = clock64();
    }
    if (w.phase == PH_OUT) continue;  // the other end may go out too
    if (HET) status = CTL_EVAL;
    break;
  }
  if (lane == 0) {
    ch.pending = pend;
    P.pending[c] = pend;
  }
  wc_store(ch, w, lane);
  if (prof) {
    g->c_result += acc_res;
    g->c_step += acc_step;
    g->c_prop += acc_prop;
    g->c_free += acc_free;
    g->c_setup += acc_setup;
    g->n_free += cnt_free;
    g->n_setup += cnt_setup;
    g->n_step += cnt_step;
  }
  return w.done && status == CTL_AGAIN ? CTL_WAIT : status;
}

template <int NDET>
__device__ __forceinline__ void flow_control_warp(const LikeConst& L, const SamplerConst& S, const DeviceBuffers& B,
                                                  const SamplerPtrs& P, int c, ChainState& ch, EvalRecord& rx,
                                                  int lane) {
  control_step_warp<NDET, false>(L, S, B, P, c, ch, rx, lane);
}

template <int NDET, bool MIXED>
__global__ void __launch_bounds__(kFlowThreads, 1)
    k_ns_flow(LikeConst L, SamplerConst S, DeviceBuffers B, SamplerPtrs P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int slice = blockIdx.x;
  const int b0 = B.slice_begin[slice], b1 = B.slice_begin[slice + 1];
  const int nb = b1 - b0;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  NSGlobal* g = P.g;

  // slice-resident data (mixed precision): D_i and the tile of each bin, then
  // the slice's tile table and one anchor row per warp (so that crossing into
  // a tile in the bin loop reads shared memory, not L2)
  float2* s_data = reinterpret_cast<float2*>(smem);
  int* s_tile = reinterpret_cast<int*>(s_data + (size_t)NDET * nb);
  size_t fixed_bytes = 0;
  TileInfo* s_ti = nullptr;
  float* s_anc = nullptr;
  int tf = 0;
  if (MIXED) {
    for (int i = 0; i < NDET; ++i)
      for (int kq = tid; kq < nb; kq += blockDim.x) s_data[i * nb + kq] = B.data32[(size_t)i * L.n_bins + b0 + kq];
    for (int kq = tid; kq < nb; kq += blockDim.x) s_tile[kq] = B.bin_tile[b0 + kq];
    fixed_bytes = (((size_t)nb * (NDET * sizeof(float2) + sizeof(int))) + 15) & ~(size_t)15;
    s_ti = reinterpret_cast<TileInfo*>(smem + fixed_bytes);
    s_anc = reinterpret_cast<float*>(smem + fixed_bytes + flow_tile_bytes(S.max_tiles_slice, 0));
    fixed_bytes += flow_tile_bytes(S.max_tiles_slice, kFlowThreads / 32);
    tf = B.bin_tile[b0];
    const int nt = B.bin_tile[b1 - 1] - tf + 1;
    for (int t = tid; t < nt; t += blockDim.x) s_ti[t] = B.tiles[tf + t];
  }
  __syncthreads();
  unsigned char* dyn = smem + fixed_bytes;  // per-warp records, or sort buffers (boundary)
  EvalRecord* rec = reinterpret_cast<EvalRecord*>(dyn) + warp;
  int* s_claim = reinterpret_cast<int*>(dyn + S.claim_off);  // per request slot: units this CTA has taken
  float* const arow = MIXED ? s_anc + (size_t)warp * S.max_tiles_slice * kAnchorStride : nullptr;
  const int G = S.flow_parts;
  const int target = S.n_ctas * G;  // units per request: G parts of every slice

  const bool timer = blockIdx.x == 0 && tid == 0;
  unsigned long long t0 = gtimer(), t1;
  for (;;) {
    if (!grid_sync(g, S.n_ctas, S.spin_limit)) return;
    if (timer) {
      t1 = gtimer();
      g->t_wait_sweep += t1 - t0;
      t0 = t1;
      g->rounds += 1;
    }
    if (blockIdx.x == 0) ns_boundary(L, S, P, dyn);
    for (int c = tid; c < S.n_slots; c += blockDim.x) s_claim[c] = 0;
    if (!grid_sync(g, S.n_ctas, S.spin_limit)) return;
    if (timer) {
      t1 = gtimer();
      g->t_bound += t1 - t0;
      t0 = t1;
    }
    if (*(volatile int*)&g->status != ST_RUNNING) return;

    long long idle = 0;
    unsigned long long my_units = 0, my_unit_cyc = 0, my_idle_cyc = 0, my_ctrl_cyc = 0;
    long long tpoll = clock64();
    if (warp == 0) {
      // ---- control of the chains homed on this CTA.  Mixed precision: the
      // chains' state and current-point records stay in this CTA's shared
      // memory for the iteration (warp-parallel control); FP64: in global
      // memory, one lane.  A chain is ready when every CTA finished its request
      ChainState* hs = reinterpret_cast<ChainState*>(dyn + S.ctl_off);
      EvalRecord* hr = reinterpret_cast<EvalRecord*>(hs + S.ctl_slots);
      if (MIXED) {
        for (int c = blockIdx.x, i = 0; c < S.nrep; c += S.n_ctas, ++i) {
          warp_copy_cg(&hs[i], &P.chains[c], sizeof(ChainState), lane);
          warp_copy_cg(&hr[i], &P.recx[c], sizeof(EvalRecord), lane);
        }
      }
      for (;;) {
        bool all_done = true, progressed = false;
        for (int c = blockIdx.x, i = 0; c < S.nrep; c += S.n_ctas, ++i) {
          int st = 0;  // 0 done, 1 waiting, 2 ready
          if (lane == 0) {
            const ChainState* ch = MIXED ? &hs[i] : &P.chains[c];
            const int pm = ch->pending;  // bit 0: slot c, bit 1: slot nrep + c (two-ended stepping-out)
            if (ch->done)
              st = 0;
            else if (pm)
              st = ((pm & 1) && ld_acquire(&P.done_cnt[c]) >= target) ||
                           ((pm & 2) && ld_acquire(&P.done_cnt[S.nrep + c]) >= target)
                       ? 2
                       : 1;
            else
              st = 2;
          }
          st = __shfl_sync(0xffffffffu, st, 0);
          if (st == 0) continue;
          all_done = false;
          if (st == 1) continue;
          progressed = true;
          const long long tc0 = clock64();
          if (MIXED)
            flow_control_warp<NDET>(L, S, B, P, c, hs[i], hr[i], lane);
          else
            flow_control<NDET, MIXED>(L, S, B, P, c, lane);
          my_ctrl_cyc += clock64() - tc0;
        }
        if (all_done) break;
        if (*(volatile int*)&g->error) break;
        if (progressed) {
          idle = 0;
        } else {
          if (++idle > S.spin_limit) {
            if (lane == 0) atomicCAS(&g->error, 0, SWIG_E_TIMEOUT);
            break;
          }
          __nanosleep(64);
        }
      }
      if (MIXED)
        for (int c = blockIdx.x, i = 0; c < S.nrep; c += S.n_ctas, ++i)
          warp_copy(&P.chains[c], &hs[i], sizeof(ChainState), lane);
    } else {
      // ---- sweep: claim (chain, request, part) units, lowest chain first,
      // and evaluate that part of this CTA's slice, one warp per unit (the G
      // parts of a request may run on G warps at once)
      for (;;) {
        if (*(volatile int*)&g->chains_done >= S.nrep) break;
        if (*(volatile int*)&g->error) break;
        // s_claim[c] = units of chain c this CTA has taken: request r owns
        // units (r - 1) G .. r G - 1, one per part
        int cc = -1, part = 0;
        int rq[4];  // request words of four groups of 32 slots, read together
        for (int base = 0; base < S.n_slots && cc < 0; base += 32) {
          const int c = base + lane;
          const int gq = (base >> 5) & 3;
          if (gq == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              rq[q] = base + 32 * q + lane < S.n_slots ? *(volatile int*)&P.req[base + 32 * q + lane] : 0;
          }
          int r = 0;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q == gq) r = rq[q] >> 3;
          bool cand = false;
          if (c < S.n_slots) cand = r * G > *(volatile int*)&s_claim[c];
          unsigned m = __ballot_sync(0xffffffffu, cand);
          while (m) {
            const int leader = __ffs(m) - 1;
            int won = 0, pt = 0;
            if (lane == leader) {
              const int old = *(volatile int*)&s_claim[c];
              if (old < r * G) {
                const int nv = max(old, (r - 1) * G) + 1;
                won = atomicCAS(&s_claim[c], old, nv) == old;
                pt = nv - 1 - (r - 1) * G;
              }
            }
            if (__shfl_sync(0xffffffffu, won, leader)) {
              cc = base + leader;
              part = __shfl_sync(0xffffffffu, pt, leader);
              break;
            }
            m &= ~(1u << leader);
          }
        }
        if (cc < 0) {
          if (++idle > S.spin_limit) {
            if (lane == 0) atomicCAS(&g->error, 0, SWIG_E_TIMEOUT);
            break;
          }
          __nanosleep(100);
          continue;
        }
        idle = 0;
        const long long tu0 = clock64();
        my_idle_cyc += tu0 - tpoll;
        __threadfence();  // acquire: the request word was read relaxed
        load_record_cg<MIXED>(&B.rec[cc], rec, lane);
        {
          const int lo = (int)(((long long)nb * part) / G), hi = (int)(((long long)nb * (part + 1)) / G);
          const size_t pidx = (((size_t)cc * L.n_slices + slice) * G + part) * kPartialStride;
          if (MIXED) {
            float* row = arow;
            if (hi > lo) {
              const int t_lo = s_tile[lo] - tf, t_hi = s_tile[hi - 1] - tf;
              for (int t = t_lo + lane; t <= t_hi; t += 32)
                compute_anchor(NDET, s_ti[t], B.basis[tf + t], *rec, row + (size_t)t * kAnchorStride);
            }
            __syncwarp();
            float v[2 * NDET];
            sweep_warp_mixed<NDET>(L, s_data, nb, s_tile, b0, lo, hi, s_ti, row, tf, *rec, lane, v);
#pragma unroll
            for (int j = 0; j < 2 * NDET; ++j)
              if (lane == j) B.partials32[pidx + j] = v[j];
          } else {
            double v[2 * NDET];
            sweep_warp_fp64<NDET>(L, B.data64, B.ftab, b0 + lo, b0 + hi, *rec, lane, v);
#pragma unroll
            for (int j = 0; j < 2 * NDET; ++j)
              if (lane == j) B.partials64[pidx + j] = v[j];
          }
        }
        __syncwarp();
        if (lane == 0) red_release_add(&P.done_cnt[cc], 1);
        tpoll = clock64();
        my_units += 1;
        my_unit_cyc += tpoll - tu0;
      }
    }
    my_idle_cyc += clock64() - tpoll;
    if (blockIdx.x == 0 && lane == 0) {
      atomicAdd(&g->f_units, my_units);
      atomicAdd(&g->f_unit_cyc, my_unit_cyc);
      atomicAdd(&g->f_idle_cyc, my_idle_cyc);
    }
    if (lane == 0 && P.cta_prof) {
      unsigned long long* cp = P.cta_prof + 4 * (size_t)blockIdx.x;
      if (warp == 0) {
        atomicAdd(cp + 3, my_ctrl_cyc);
      } else {
        atomicAdd(cp + 0, my_units);
        atomicAdd(cp + 1, my_unit_cyc);
        atomicAdd(cp + 2, my_idle_cyc);
      }
    }
    __syncthreads();
    if (timer) {
      t1 = gtimer();
      g->t_ctrl += t1 - t0;
      t0 = t1;
    }
  }
}

// ---------------------------------------------------------------------------
// Several events in one persistent launch (an injection campaign): every CTA
// holds its slice of each event's grid in shared memory, the control warps
// serve chains of all events, the sweep warps claim requests of any event.
// Each event keeps its own NS state and boundary (run by CTA e for event e);
// the grid meets around the boundaries, and the launch returns as soon as any
// event leaves the running state, before any event starts new chains, so that
// the others resume exactly where they stopped.  Per event the arithmetic and
// its order are those of k_ns_flow: the results equal separate runs.
// ---------------------------------------------------------------------------
struct EventDesc {
  LikeConst L;
  SamplerConst S;
  DeviceBuffers B;
  SamplerPtrs P;
  int smem_off;  // byte offset of the event's slice data in the CTA's shared memory
};

template <int NDET>
__global__ void __launch_bounds__(kFlowThreads, 1)
    k_ns_multi(const EventDesc* __restrict__ ev, int n_ev, NSGlobal* gb, int n_ctrl, int dyn_off, int ctl_off,
               int ctl_slots) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_claim[kMaxChains];  // [event][chain]: units this CTA has taken (see k_ns_flow)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = ev[0].S.nrep;
  const int G = ev[0].S.flow_parts;
  const long long spin_limit = ev[0].S.spin_limit;
  for (int e = 0; e < n_ev; ++e) {
    const LikeConst& L = ev[e].L;
    if ((int)blockIdx.x >= L.n_slices) continue;
    const int b0 = ev[e].B.slice_begin[blockIdx.x], nb = ev[e].B.slice_begin[blockIdx.x + 1] - b0;
    float2* sd = reinterpret_cast<float2*>(smem + ev[e].smem_off);
    int* stile = reinterpret_cast<int*>(sd + (size_t)NDET * nb);
    for (int i = 0; i < NDET; ++i)
      for (int kq = tid; kq < nb; kq += blockDim.x) sd[i * nb + kq] = ev[e].B.data32[(size_t)i * L.n_bins + b0 + kq];
    for (int kq = tid; kq < nb; kq += blockDim.x) stile[kq] = ev[e].B.bin_tile[b0 + kq];
  }
  __syncthreads();
  unsigned char* dyn = smem + dyn_off;
  EvalRecord* rec = reinterpret_cast<EvalRecord*>(dyn) + warp;
  for (;;) {
    if (!grid_sync(gb, gridDim.x, spin_limit)) return;
    if ((int)blockIdx.x < n_ev) ns_boundary_check(ev[blockIdx.x].L, ev[blockIdx.x].S, ev[blockIdx.x].P, dyn);
    if (!grid_sync(gb, gridDim.x, spin_limit)) return;
    bool all_run = true;
    for (int e = 0; e < n_ev; ++e) all_run = all_run && *(volatile int*)&ev[e].P.g->status == ST_RUNNING;
    if (!all_run) return;
    if ((int)blockIdx.x < n_ev) ns_boundary_advance(ev[blockIdx.x].L, ev[blockIdx.x].S, ev[blockIdx.x].P, dyn);
    for (int q = tid; q < n_ev * k; q += blockDim.x) s_claim[q] = 0;
    if (!grid_sync(gb, gridDim.x, spin_limit)) return;

    long long idle = 0;
    if (warp < n_ctrl) {
      // ---- control of the chains homed on (this CTA, this warp): warp-
      // parallel, with their state in this warp's shared-memory slots
      ChainState* hs = reinterpret_cast<ChainState*>(smem + ctl_off) + (size_t)warp * ctl_slots;
      EvalRecord* hr = reinterpret_cast<EvalRecord*>(reinterpret_cast<ChainState*>(smem + ctl_off) +
                                                     (size_t)n_ctrl * ctl_slots) + (size_t)warp * ctl_slots;
      for (int q = blockIdx.x + gridDim.x * warp, i = 0; q < n_ev * k; q += gridDim.x * n_ctrl, ++i) {
        const EventDesc& E = ev[q / k];
        warp_copy_cg(&hs[i], &E.P.chains[q % k], sizeof(ChainState), lane);
        warp_copy_cg(&hr[i], &E.P.recx[q % k], sizeof(EvalRecord), lane);
      }
      for (;;) {
        bool all_done = true, progressed = false;
        for (int q = blockIdx.x + gridDim.x * warp, i = 0; q < n_ev * k; q += gridDim.x * n_ctrl, ++i) {
          const EventDesc& E = ev[q / k];
          const int c = q % k;
          int st = 0;  // 0 done, 1 waiting, 2 ready
          if (lane == 0) {
            const ChainState* ch = &hs[i];
            if (ch->done)
              st = 0;
            else if (ch->pending)
              st = ld_acquire(&E.P.done_cnt[c]) >= E.L.n_slices * G ? 2 : 1;
            else
              st = 2;
          }
          st = __shfl_sync(0xffffffffu, st, 0);
          if (st == 0) continue;
          all_done = false;
          if (st == 1) continue;
          progressed = true;
          flow_control_warp<NDET>(E.L, E.S, E.B, E.P, c, hs[i], hr[i], lane);
        }
        if (all_done) break;
        if (*(volatile int*)&gb->error) break;
        if (progressed) {
          idle = 0;
        } else {
          if (++idle > spin_limit) {
            if (lane == 0) atomicCAS(&gb->error, 0, SWIG_E_TIMEOUT);
            break;
          }
          __nanosleep(64);
        }
      }
      for (int q = blockIdx.x + gridDim.x * warp, i = 0; q < n_ev * k; q += gridDim.x * n_ctrl, ++i)
        warp_copy(&ev[q / k].P.chains[q % k], &hs[i], sizeof(ChainState), lane);
    } else {
      // ---- sweep: claim (event, chain, request, part) units and evaluate
      // that part of this CTA's slice of the event
      for (;;) {
        bool over = true;
        for (int e = 0; e < n_ev; ++e) over = over && *(volatile int*)&ev[e].P.g->chains_done >= k;
        if (over) break;
        if (*(volatile int*)&gb->error) break;
        int qq = -1, part = 0;
        for (int base = 0; base < n_ev * k && qq < 0; base += 32) {
          const int q = base + lane;
          int r = 0;
          bool cand = false;
          if (q < n_ev * k && (int)blockIdx.x < ev[q / k].L.n_slices) {
            r = (*(volatile int*)&ev[q / k].P.req[q % k]) >> 3;
            cand = r * G > *(volatile int*)&s_claim[q];
          }
          unsigned msk = __ballot_sync(0xffffffffu, cand);
          while (msk) {
            const int leader = __ffs(msk) - 1;
            int won = 0, pt = 0;
            if (lane == leader) {
              const int old = *(volatile int*)&s_claim[q];
              if (old < r * G) {
                const int nv = max(old, (r - 1) * G) + 1;
                won = atomicCAS(&s_claim[q], old, nv) == old;
                pt = nv - 1 - (r - 1) * G;
              }
            }
            if (__shfl_sync(0xffffffffu, won, leader)) {
              qq = base + leader;
              part = __shfl_sync(0xffffffffu, pt, leader);
              break;
            }
            msk &= ~(1u << leader);
          }
        }
        if (qq < 0) {
          if (++idle > spin_limit) {
            if (lane == 0) atomicCAS(&gb->error, 0, SWIG_E_TIMEOUT);
            break;
          }
          __nanosleep(100);
          continue;
        }
        idle = 0;
        const EventDesc& E = ev[qq / k];
        const int cc = qq % k;
        const int slice = blockIdx.x;
        const int b0 = E.B.slice_begin[slice], nb = E.B.slice_begin[slice + 1] - b0;
        const float2* sd = reinterpret_cast<const float2*>(smem + E.smem_off);
        const int* stile = reinterpret_cast<const int*>(sd + (size_t)NDET * nb);
        const int tf = stile[0];
        // the parts of a request may run on several warps: each fills the
        // anchors of its own tiles (a tile shared by two parts gets the same
        // values from both)
        float* row = E.P.anchor_buf + ((size_t)slice * k + cc) * E.S.max_tiles_slice * kAnchorStride;
        const int lo = (int)(((long long)nb * part) / G), hi = (int)(((long long)nb * (part + 1)) / G);
        __threadfence();  // acquire: the request word was read relaxed
        load_record_cg(&E.B.rec[cc], rec, lane);
        if (hi > lo)
          for (int t = stile[lo] - tf + lane; t <= stile[hi - 1] - tf; t += 32)
            compute_anchor(NDET, E.B.tiles[tf + t], E.B.basis[tf + t], *rec, row + (size_t)t * kAnchorStride);
        __syncwarp();
        float v[2 * NDET];
        sweep_warp_mixed<NDET>(E.L, sd, nb, stile, b0, lo, hi, E.B.tiles + tf, row, tf, *rec, lane, v);
        const size_t pidx = (((size_t)cc * E.L.n_slices + slice) * G + part) * kPartialStride;
#pragma unroll
        for (int j = 0; j < 2 * NDET; ++j)
          if (lane == j) E.B.partials32[pidx + j] = v[j];
        __syncwarp();
        if (lane == 0) red_release_add(&E.P.done_cnt[cc], 1);
      }
    }
    __syncthreads();
  }
}

// Persistent sampler for the heterodyned likelihood (Sec. 3.4).  A
// heterodyned evaluation is a few hundred to a few thousand bins, so one CTA
// owns one chain at a time.  Warp 0 runs the chain's control with the same
// warp-parallel code as the full-grid sampler (state in this CTA's shared
// memory), sets up the proposal's record and forms the per-evaluation
// constants of the contraction (coefficient and delay differences from the
// fiducial, C_i / C0_i; one per lane) in shared memory; then every warp
// contracts a share of the bins (31-bin chunks, strided by warp), the
// per-warp sums are added in warp order (double-float), and warp 0 forms the
// epilogue and the per-detector cache with one detector per lane.  The
// chains of one NS iteration run independently to completion; the grid meets
// only at the iteration boundary.  Projection-only blocks (d_L, iota, psi,
// phi_c) reuse each chain's per-detector cache of its last full evaluation,
// as on the full grid.  With t_c marginalised the bin pass also stores the
// edge products y_e in shared memory (the boundary's scratch, unused between
// boundaries) and the warps then share the time grid's 32-node chunks
// (het.cuh tm_pass); there are no projection-only blocks in that mode.
template <int NDET>
__device__ __forceinline__ void het_prepare_warp(const LikeConst& L, const HetTables& H, const EvalRecord& r,
                                                 HetPrep<NDET>& p, int lane) {
  const EvalRecord& f0 = *H.fid;
  if (lane < NBASIS) p.dc[lane] = df_from_double(r.c[lane] - f0.c[lane]);
  if (lane >= 16 && lane < 16 + NDET) {
    const int i = lane - 16;
    p.dtau[i] = df_from_double(r.tau[i] - f0.tau[i]);
    const double iden = L.het_fid_iden[i];
    p.rho_re[i] = (float)((r.cre[i] * f0.cre[i] + r.cim[i] * f0.cim[i]) * iden);
    p.rho_im[i] = (float)((r.cim[i] * f0.cre[i] - r.cre[i] * f0.cim[i]) * iden);
  }
  __syncwarp();
}

template <int NDET>
__global__ void __launch_bounds__(kHetThreads, 1)
    k_ns_het(LikeConst L, SamplerConst S, DeviceBuffers B, SamplerPtrs P) {
  static_assert(sizeof(HetStage<NDET>) == (size_t)NDET * 32 * (16 + 8) + 2 * 32 * 4, "stage layout (kernels.h)");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float s_sum[kHetThreads / 32][3 * NDET];
  __shared__ float s_tm[kHetThreads / 32][2];
  __shared__ HetPrep<NDET> s_prep;
  __shared__ int s_st;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_warps = blockDim.x >> 5;
  NSGlobal* g = P.g;
  const HetTables H = het_tables(B);
  const int nc = het_chunks(H.n_bins);
  ChainState& ch = *reinterpret_cast<ChainState*>(smem + S.ctl_off);
  EvalRecord& rx = *reinterpret_cast<EvalRecord*>(smem + S.ctl_off + sizeof(ChainState));
  float* s_anc = reinterpret_cast<float*>(smem + S.claim_off);  // [chunks][kHetAncStride]
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  unsigned long long t0 = gtimer(), t1;
  // per-CTA cycle counters: contractions, cycles in them (bin pass, time
  // pass, reductions), cycles the other warps wait on warp 0 (control,
  // epilogue), and warp 0's cycles in control
  // (shared memory, one writer each: warp 1's lane 0 and warp 0's lane 0)
  __shared__ unsigned long long s_prof[5];
  if (threadIdx.x < 5) s_prof[threadIdx.x] = 0;
  const bool t_sw = warp == 1 && lane == 0, t_ct = warp == 0 && lane == 0;
  for (;;) {
    if (!grid_sync(g, S.n_ctas, S.spin_limit)) return;
    if (timer) {
      t1 = gtimer();
      g->t_wait_sweep += t1 - t0;
      t0 = t1;
      g->rounds += 1;
    }
    if (blockIdx.x == 0) ns_boundary(L, S, P, smem);
    if (!grid_sync(g, S.n_ctas, S.spin_limit)) return;
    if (timer) {
      t1 = gtimer();
      g->t_bound += t1 - t0;
      t0 = t1;
    }
    if (*(volatile int*)&g->status != ST_RUNNING) return;
    if (L.tm_M > 0) {  // the boundary may have used the scratch: twiddles again
      tm_load_twiddles(L, H, smem, H.n_bins);
      __syncthreads();
    }
    for (int c = blockIdx.x; c < S.nrep; c += gridDim.x) {
      // warp 0's copy of the last evaluation's result (see control_step_warp)
      double ly = 0.0, kapc = 0.0, vvc = 0.0;
      if (warp == 0) {
        warp_copy_cg(&ch, &P.chains[c], sizeof(ChainState), lane);
        warp_copy_cg(&rx, &P.recx[c], sizeof(EvalRecord), lane);
      }
      if (t_sw) s_prof[4] = clock64();
      for (long long guard = 0; guard < (1ll << 24); ++guard) {
        if (warp == 0) {
          const long long tc = clock64();
          const int st = control_step_warp<NDET, true>(L, S, B, P, c, ch, rx, lane, ly, kapc, vvc);
          if (st == CTL_EVAL) het_prepare_warp<NDET>(L, H, B.rec[c], s_prep, lane);
          if (lane == 0) s_st = st;
          if (t_ct) s_prof[3] += clock64() - tc;
        }
        __syncthreads();
        if (t_sw) {
          const unsigned long long tu = clock64();
          s_prof[2] += tu - s_prof[4];
          s_prof[4] = tu;
        }
        const int st = s_st;
        if (st == CTL_WAIT) break;    // the chain is done
        if (st == CTL_AGAIN) continue;  // projection-only budget used up
        const EvalRecord& r = B.rec[c];
        const bool valid = r.valid != 0;
        float zr[NDET], zi[NDET], hh[NDET];
#pragma unroll
        for (int i = 0; i < NDET; ++i) zr[i] = zi[i] = hh[i] = 0.0f;
        if (valid) {  // block-uniform
          const HetPrep<NDET>& p = s_prep;  // read from shared memory where used
          // chunk anchors, one thread per chunk, then the edge pass
          for (int q = threadIdx.x; q < nc; q += blockDim.x) het_anchor<NDET>(H, p, q, s_anc + q * kHetAncStride);
          __syncthreads();
          unsigned char* stage =
              S.stage_off > 0 ? smem + S.stage_off + (size_t)warp * 2 * sizeof(HetStage<NDET>) : nullptr;
          if (L.tm_n > 0)
            het_chunks_warp<NDET, true>(H, p, s_anc, warp, n_warps, lane, stage, zr, zi, hh,
                                        reinterpret_cast<float2*>(smem));
          else
            het_chunks_warp<NDET>(H, p, s_anc, warp, n_warps, lane, stage, zr, zi, hh);
          het_warp_reduce<NDET>(zr, zi, hh);
        }
        if (lane == 0) {
#pragma unroll
          for (int i = 0; i < NDET; ++i) {
            s_sum[warp][3 * i] = zr[i];
            s_sum[warp][3 * i + 1] = zi[i];
            s_sum[warp][3 * i + 2] = hh[i];
          }
        }
        __syncthreads();
        if (L.tm_n > 0 && valid) {  // block-uniform
          float wm, ws;
          if (L.tm_M > 0)
            tm_pass_nufft(L, H, reinterpret_cast<float2*>(smem), tm_nufft_grid(smem, H.n_bins),
                          tm_nufft_tw(smem, H.n_bins, L.tm_M), warp, n_warps, lane,
                          nullptr, wm, ws);
          else
            tm_pass(L, H, reinterpret_cast<const float2*>(smem), warp, n_warps, lane, nullptr, wm, ws);
          if (lane == 0) {
            s_tm[warp][0] = wm;
            s_tm[warp][1] = ws;
          }
          __syncthreads();
        }
        if (t_sw) {
          const unsigned long long tw = clock64();
          s_prof[0] += 1;
          s_prof[1] += tw - s_prof[4];
          s_prof[4] = tw;
        }
        if (warp == 0) {
          // lane i < NDET: detector i's sums over the warps in warp order
          // (double-float), its cache entries, then the network epilogue
          double dz_r = 0.0, dz_i = 0.0, dhh = 0.0;
          if (lane < NDET) {
            dfl a = {0.0f, 0.0f}, b = {0.0f, 0.0f}, h = {0.0f, 0.0f};
            for (int w = 0; w < n_warps; ++w) {
              a = df_add(a, dfl{s_sum[w][3 * lane], 0.0f});
              b = df_add(b, dfl{s_sum[w][3 * lane + 1], 0.0f});
              h = df_add(h, dfl{s_sum[w][3 * lane + 2], 0.0f});
            }
            dz_r = (double)a.hi + (double)a.lo;
            dz_i = (double)b.hi + (double)b.lo;
            dhh = (double)h.hi + (double)h.lo;
          }
          double k2[2] = {0.0, 0.0}, vi = 0.0;
          if (lane < NDET && valid) het_cache(L, r, lane, dz_r, dz_i, dhh, k2, &vi);
          // component j of the cache on lane j, detector i's vv on lane i
          const double k0 = __shfl_sync(kFull, k2[0], lane < 2 * NDET ? lane >> 1 : 0);
          const double k1 = __shfl_sync(kFull, k2[1], lane < 2 * NDET ? lane >> 1 : 0);
          kapc = lane < 2 * NDET ? ((lane & 1) ? k1 : k0) : 0.0;
          vvc = lane < NDET ? vi : 0.0;
          double Z_re = 0.0, Z_im = 0.0, HH = 0.0;
#pragma unroll
          for (int i = 0; i < NDET; ++i) {
            Z_re += __shfl_sync(kFull, dz_r, i);
            Z_im += __shfl_sync(kFull, dz_i, i);
            HH += __shfl_sync(kFull, dhh, i);
          }
          double out = -INFINITY;
          if (lane == 0 && valid) out = L.tm_n > 0 ? tm_finish(L, s_tm, n_warps, HH) : het_epilogue(L, Z_re, Z_im, HH);
          ly = __shfl_sync(kFull, out, 0);
          if (!valid) kapc = vvc = 0.0;
        }
      }
      if (warp == 0) warp_copy(&P.chains[c], &ch, sizeof(ChainState), lane);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (blockIdx.x == 0) {
        g->f_units += s_prof[0];
        g->f_unit_cyc += s_prof[1];
        g->f_idle_cyc += s_prof[2];
      }
      if (P.cta_prof) {
        unsigned long long* cp = P.cta_prof + 4 * (size_t)blockIdx.x;
        for (int j = 0; j < 4; ++j) cp[j] += s_prof[j];
      }
      for (int j = 0; j < 4; ++j) s_prof[j] = 0;
    }
    if (timer) {
      t1 = gtimer();
      g->t_ctrl += t1 - t0;
      t0 = t1;
    }
  }
}

// Initial live set: m unit-cube draws (Philox, stream tag 2) and their theta.
__global__ void k_init_live(SamplerConst S, double* live_u, double* theta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.nlive) return;
  double u[kMaxDim];
  for (int j = 0; j < S.ndim; ++j) {
    const uint4 r = philox4x32_10(make_uint4((unsigned)j, (unsigned)i, 0xFFFFFFFFu, 2u), S.key0, S.key1);
    u[j] = u01_from(r);
    live_u[(size_t)i * S.ndim + j] = u[j];
  }
  prior_map(S.prior, u, theta + (size_t)i * SWIG_N_PARAMS, &S.sky);
}

__global__ void k_dead_theta(SamplerConst S, const double* u, int n, double* theta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) prior_map(S.prior, u + (size_t)i * S.ndim, theta + (size_t)i * SWIG_N_PARAMS, &S.sky);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct SamplerState {
  SamplerPtrs P = {};
  double* harm = nullptr;
  double* lw = nullptr;
  double* init_theta = nullptr;
  float* anchor_buf = nullptr;
  unsigned long long* cta_prof = nullptr;  // [n_ctas][4]
  int cta_prof_n = 0;
  int cap_iters = 0;
  int nlive = 0, nrep = 0, ndim = 0;
};

namespace {

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void release(SamplerState* s) {
  if (!s) return;
  dfree(s->P.live_u);
  dfree(s->P.live_logl);
  dfree(s->P.live_kap);
  dfree(s->P.live_vv);
  dfree(s->P.chains);
  dfree(s->P.recx);
  dfree(s->P.pending);
  dfree(s->P.req);
  dfree(s->P.done_cnt);
  dfree(s->P.chol);
  dfree(s->P.g);
  dfree(s->P.dead_u);
  dfree(s->P.dead_logl);
  dfree(s->P.dead_logw);
  dfree(s->harm);
  dfree(s->lw);
  dfree(s->init_theta);
  dfree(s->anchor_buf);
  dfree(s->cta_prof);
}

int fail(swig_ctx* c, int code, const std::string& m) {
  c->err = m;
  return code;
}

#define SCUDA(call)                                                                                        \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess)                                                                                 \
      return fail(c, e_ == cudaErrorMemoryAllocation ? SWIG_E_NOMEM : SWIG_E_CUDA,                         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                                     \
  } while (0)

template <int NDET, bool MIXED>
void* kernel_ptr() {
  return (void*)k_ns_flow<NDET, MIXED>;
}

void* pick_kernel(int n_det, bool mixed) {
  if (mixed) {
    switch (n_det) {
      case 1: return kernel_ptr<1, true>();
      case 2: return kernel_ptr<2, true>();
      case 3: return kernel_ptr<3, true>();
      default: return kernel_ptr<4, true>();
    }
  }
  switch (n_det) {
    case 1: return kernel_ptr<1, false>();
    case 2: return kernel_ptr<2, false>();
    case 3: return kernel_ptr<3, false>();
    default: return kernel_ptr<4, false>();
  }
}

void* pick_multi_kernel(int n_det) {
  switch (n_det) {
    case 1: return (void*)k_ns_multi<1>;
    case 2: return (void*)k_ns_multi<2>;
    case 3: return (void*)k_ns_multi<3>;
    default: return (void*)k_ns_multi<4>;
  }
}

void* pick_het_kernel(int n_det) {
  switch (n_det) {
    case 1: return (void*)k_ns_het<1>;
    case 2: return (void*)k_ns_het<2>;
    case 3: return (void*)k_ns_het<3>;
    default: return (void*)k_ns_het<4>;
  }
}

}  // namespace
}  // namespace swig

using namespace swig;

void swig_sampler_release(swig_ctx* c) {
  if (c && c->sampler) {
    release(c->sampler);
    delete c->sampler;
    c->sampler = nullptr;
  }
}

extern "C" {

int swig_set_wait_limit(swig_ctx* c, long long spins) {
  if (!c) return SWIG_E_ARG;
  if (spins < 0) return fail(c, SWIG_E_ARG, "wait limit must be >= 0");
  c->wait_limit = spins;
  return SWIG_OK;
}

}  // extern "C"

namespace swig {
namespace {

// Host state of one sampler run between its set-up and its result.
struct RunState {
  SamplerConst S;
  SamplerState* st = nullptr;
  size_t smem = 0, fixed = 0, tail = 0;  // tail: per-warp records / sort buffers (multi-event layout)
  void* kern = nullptr;
  int threads = 0;
  bool het = false, mixed = false, learned = false;
  int m = 0, k = 0, nd = 0;
  float learn_lr = 0.0f;
  int learn_steps = 0;
  std::vector<double> du, dl, dw;
  NSGlobal gh;
  long long total_iters = 0;
  double persistent_ms = 0.0, learn_ms = 0.0;
  long long persistent_launches = 0, learn_rounds = 0;
  bool finished = false;
  std::chrono::steady_clock::time_point t_start;
};

}  // namespace
}  // namespace swig

using namespace swig;

namespace {

// Validation, preparation, sampler constants, buffers, the initial live set
// and the NS state: everything before the first persistent launch.
int run_setup(swig_ctx* c, RunState& R) {
  if (!c->prior_set) return fail(c, SWIG_E_STATE, "prior not set");
  if (!c->cfg_set) return fail(c, SWIG_E_STATE, "sampler not configured");
  if (c->cfg.nlive > kMaxSort) return fail(c, SWIG_E_ARG, "nlive must be <= 8192 for the device sort");
  if (c->cfg.nrep > kMaxChains) return fail(c, SWIG_E_ARG, "nrep must be <= 2048");
  int rc = prepare(c);
  if (rc) return rc;
  R.t_start = std::chrono::steady_clock::now();
  const bool het = c->prepared_like == SWIG_LIKE_HET;
  const bool mixed = !het && c->prepared_precision == SWIG_PREC_MIXED;
  R.het = het;
  R.mixed = mixed;
  const int m = c->cfg.nlive, k = c->cfg.nrep;
  R.m = m;
  R.k = k;
  const LikeConst& L = c->L;
  if (!het && k > 32 * L.n_slices) return fail(c, SWIG_E_ARG, "nrep exceeds 32 chains per CTA");
  const int het_ctas = std::max(1, std::min(c->sm_count, k));

  SamplerConst& S = R.S;
  std::memset(&S, 0, sizeof(S));
  S.nlive = m;
  S.nrep = k;
  S.sweeps = c->cfg.sweeps;
  S.steps_per_dim = c->cfg.steps_per_dim;
  S.dlogz = c->cfg.dlogz;
  S.key0 = (unsigned)(c->cfg.seed & 0xFFFFFFFFu);
  S.key1 = (unsigned)(c->cfg.seed >> 32);
  S.mixed = mixed ? 1 : 0;
  S.n_ctas = het ? het_ctas : L.n_slices;
  S.het = het ? 1 : 0;
  S.spin_limit = c->wait_limit;
  if ((rc = make_sky_frame(c, &S.sky))) return rc;
  int nd = 0;
  for (int i = 0; i < SWIG_N_PARAMS; ++i) {
    const swig_param& p = c->params[i];
    S.prior[i] = make_prior_slot(p.kind, p.mode, p.lo, p.hi, p.value);
    if (p.mode == SWIG_MODE_SAMPLE) S.slot_of_dim[nd++] = i;
  }
  S.ndim = nd;
  R.nd = nd;
  // Gibbs blocks in increasing block id
  int ids[kMaxDim], n_ids = 0;
  for (int j = 0; j < nd; ++j) {
    const int b = c->params[S.slot_of_dim[j]].block;
    bool seen = false;
    for (int q = 0; q < n_ids; ++q) seen = seen || ids[q] == b;
    if (!seen) ids[n_ids++] = b;
  }
  std::sort(ids, ids + n_ids);
  S.n_blocks = n_ids;
  for (int b = 0; b < n_ids; ++b) {
    S.block_size[b] = 0;
    bool free_block = true;
    int flags = 0;
    for (int j = 0; j < nd; ++j)
      if (c->params[S.slot_of_dim[j]].block == ids[b]) {
        S.block_dims[b][S.block_size[b]++] = j;
        const int slot = S.slot_of_dim[j];
        free_block = free_block && (slot == 6 || slot == 7 || slot == 8 || slot == 12);
        if (slot <= 1) flags |= BF_INTR;
        if (slot == 2 || slot == 3) flags |= BF_SPIN;
        if (slot == 4 || slot == 5) flags |= BF_TIDE;
        if (slot == 0 || slot == 6) flags |= BF_AMP;
        if (slot == 7 || slot == 8 || slot == 9 || slot == 10 || slot == 12) flags |= BF_PROJ;
        if (slot == 9 || slot == 10 || slot == 11) flags |= BF_TAU;
        if (slot == 9 || slot == 10) flags |= BF_SKY;
      }
    // time marginalisation keeps no per-detector cache at every node, so
    // projection-only blocks take the full evaluation there (and everywhere
    // when the cache is switched off)
    S.block_free[b] = (free_block && L.tm_n == 0 && !c->cfg.cache_off) ? 1 : 0;
    S.block_flags[b] = flags;
    S.block_mask[b] = 0u;
    for (int r = 0; r < S.block_size[b]; ++r) {
      S.block_mask[b] |= 1u << S.block_dims[b][r];
      S.block_rank[S.block_dims[b][r]] = r;
    }
  }
  for (int i = 0; i < SWIG_N_PARAMS; ++i) S.dim_of_slot[i] = -1;
  for (int j = 0; j < nd; ++j) S.dim_of_slot[S.slot_of_dim[j]] = j;
  S.m_pow2 = 1;
  while (S.m_pow2 < m) S.m_pow2 *= 2;
  S.max_iters = (int)std::max(1, std::min(64, c->cfg.max_iter));
  // parts per slice and request: the G parts of a request's slice are claimed
  // by up to G sweep warps of the CTA at once; each part has its own partial
  // (fixed places, fixed summation order), at most 4 (the partial buffers
  // hold 4 per slice and theta)
  S.flow_parts = c->cfg.flow_parts > 0 ? c->cfg.flow_parts : SWIG_FLOW_PARTS;
  // two-ended stepping-out: the full-grid mixed-precision dataflow kernel
  S.par_out = mixed && !c->cfg.stepout_one_end ? SWIG_PAR_OUT : 0;
  S.n_slots = S.par_out ? 2 * k : k;
  // learned proposal: retrain every learn_interval iterations (one launch each)
  R.learned = c->cfg.proposal == SWIG_PROPOSAL_LEARNED;
  const double learn_mix = c->cfg.learn_mix > 0.0 ? std::min(1.0, c->cfg.learn_mix) : 0.5;
  R.learn_lr = c->cfg.learn_lr > 0.0 ? (float)c->cfg.learn_lr : 1e-3f;
  R.learn_steps = c->cfg.learn_steps > 0 ? c->cfg.learn_steps : 50;
  const int learn_interval = c->cfg.learn_interval > 0 ? c->cfg.learn_interval : 8;
  if (R.learned) {
    if (2 * nd >= m) return fail(c, SWIG_E_ARG, "the learned proposal needs nlive > 2 x sampled dimensions");
    S.max_iters = std::min(S.max_iters, learn_interval);
    S.learn_on = 1;
    S.learn_mix = (float)learn_mix;
  }

  const int max_pieces = c->B.max_pieces;
  S.max_pieces = max_pieces;
  size_t fixed = 0;
  if (mixed) fixed = ((size_t)c->B.max_slice_bins * (L.n_det * sizeof(float2) + sizeof(int)) + 15) & ~(size_t)15;
  R.fixed = fixed;
  int max_tiles = 1;
  if (mixed) {
    std::vector<int> sb(L.n_slices + 1), bt(L.n_bins);
    SCUDA(cudaMemcpy(sb.data(), c->B.slice_begin, sizeof(int) * sb.size(), cudaMemcpyDeviceToHost));
    SCUDA(cudaMemcpy(bt.data(), c->B.bin_tile, sizeof(int) * bt.size(), cudaMemcpyDeviceToHost));
    for (int s = 0; s < L.n_slices; ++s) max_tiles = std::max(max_tiles, bt[sb[s + 1] - 1] - bt[sb[s]] + 1);
  }
  S.max_tiles_slice = max_tiles;
  // the single-event kernel also keeps the slice's tile table and anchor rows
  // in shared memory (R.fixed stays the slice data alone: the multi-event
  // kernel's layout)
  const size_t flow_tiles = mixed ? flow_tile_bytes(max_tiles, kFlowThreads / 32) : 0;
  const size_t sort_bytes = (size_t)S.m_pow2 * (sizeof(double) + sizeof(int)) + kSweepThreads * sizeof(double) +
                            (size_t)k * sizeof(double) + (kMaxDim + kMaxDim * kMaxDim) * sizeof(float) + 64;
  const size_t rec_bytes = (size_t)(kFlowThreads / 32) * sizeof(EvalRecord);
  // the homed chains' state and records of the warp-parallel control follow
  // the per-warp records / sort buffers
  // (heterodyned: one slot, after the sort buffers / time-pass edge products)
  const size_t het_scratch =
      std::max(sort_bytes, L.tm_n > 0 ? het_tm_smem_bytes(c->B.het_nb, L.tm_M, L.tm_M > 0 ? L.tm_pieces : 0) : (size_t)0);
  S.ctl_slots = mixed ? (k + L.n_slices - 1) / L.n_slices : (het ? 1 : 0);
  S.ctl_off = (int)(((het ? het_scratch : std::max(rec_bytes, sort_bytes)) + 15) & ~(size_t)15);
  R.tail = std::max(rec_bytes, sort_bytes);
  const size_t ctl_bytes = (size_t)S.ctl_slots * (sizeof(ChainState) + sizeof(EvalRecord));
  S.claim_off = (int)((S.ctl_off + ctl_bytes + 15) & ~(size_t)15);
  // (heterodyned: the per-evaluation chunk anchors at claim_off, then each
  // warp's two chunk-table stages)
  S.stage_off = (int)((S.claim_off + sizeof(float) * kHetAncStride * (size_t)c->B.het_nc + 15) & ~(size_t)15);
  R.smem = het ? S.stage_off + 2 * het_stage_bytes(L.n_det) * (kHetThreads / 32)
               : fixed + flow_tiles + S.claim_off + sizeof(int) * (size_t)S.n_slots;
  if (het && R.smem > 220 * 1024) {  // no room for the chunk-table stages: direct loads
    R.smem = S.stage_off;
    S.stage_off = 0;
  }
  if (R.smem > 220 * 1024) return fail(c, SWIG_E_ARG, "problem too large for the persistent kernel's shared memory");

  // buffers
  SamplerState* st = c->sampler;
  if (!st || st->nlive != m || st->nrep != k || st->ndim != nd || st->cap_iters < S.max_iters) {
    swig_sampler_release(c);
    st = new SamplerState();
    c->sampler = st;
    st->nlive = m;
    st->nrep = k;
    st->ndim = nd;
    st->cap_iters = S.max_iters;
    SCUDA(cudaMalloc(&st->P.live_u, sizeof(double) * m * nd));
    SCUDA(cudaMalloc(&st->P.live_logl, sizeof(double) * m));
    SCUDA(cudaMalloc(&st->P.live_kap, sizeof(double) * m * 2 * SWIG_MAX_DET));
    SCUDA(cudaMalloc(&st->P.live_vv, sizeof(double) * m * SWIG_MAX_DET));
    SCUDA(cudaMalloc(&st->P.chains, sizeof(ChainState) * k));
    SCUDA(cudaMalloc(&st->P.recx, sizeof(EvalRecord) * k));
    SCUDA(cudaMalloc(&st->P.pending, sizeof(int) * k));
    SCUDA(cudaMalloc(&st->P.req, sizeof(int) * 2 * k));  // two request slots per chain
    SCUDA(cudaMalloc(&st->P.done_cnt, sizeof(int) * 2 * k));
    SCUDA(cudaMalloc(&st->P.chol, sizeof(float) * kMaxBlocks * kMaxDim * kMaxDim));
    SCUDA(cudaMalloc(&st->P.g, sizeof(NSGlobal)));
    SCUDA(cudaMalloc(&st->P.dead_u, sizeof(double) * (size_t)S.max_iters * k * nd));
    SCUDA(cudaMalloc(&st->P.dead_logl, sizeof(double) * (size_t)S.max_iters * k));
    SCUDA(cudaMalloc(&st->P.dead_logw, sizeof(double) * (size_t)S.max_iters * k));
    SCUDA(cudaMalloc(&st->harm, sizeof(double) * (k + 1)));
    SCUDA(cudaMalloc(&st->lw, sizeof(double) * (m + 1)));
    SCUDA(cudaMalloc(&st->init_theta, sizeof(double) * m * SWIG_N_PARAMS));
    std::vector<double> harm(k + 1, 0.0), lw(m + 1, 0.0);
    for (int j = 1; j <= k; ++j) harm[j] = harm[j - 1] + 1.0 / (double)(m - (j - 1));
    for (int n = 1; n <= m; ++n) lw[n] = std::log(-std::expm1(-1.0 / (double)n));
    SCUDA(cudaMemcpy(st->harm, harm.data(), sizeof(double) * harm.size(), cudaMemcpyHostToDevice));
    SCUDA(cudaMemcpy(st->lw, lw.data(), sizeof(double) * lw.size(), cudaMemcpyHostToDevice));
    st->P.harm = st->harm;
    st->P.lw = st->lw;
  }
  R.st = st;
  st->P.piece_begin = c->B.piece_begin;
  st->P.slice_piece = c->B.slice_piece;
  dfree(st->anchor_buf);
  if (mixed) {
    SCUDA(cudaMalloc(&st->anchor_buf, sizeof(float) * kAnchorStride * (size_t)L.n_slices * k * max_tiles));
  }
  st->P.anchor_buf = st->anchor_buf;
  if (st->cta_prof_n < S.n_ctas) {
    dfree(st->cta_prof);
    SCUDA(cudaMalloc(&st->cta_prof, sizeof(unsigned long long) * 4 * S.n_ctas));
    st->cta_prof_n = S.n_ctas;
  }
  SCUDA(cudaMemsetAsync(st->cta_prof, 0, sizeof(unsigned long long) * 4 * S.n_ctas, c->stream));
  st->P.cta_prof = st->cta_prof;
  st->P.learn_out = nullptr;
  if (R.learned) {
    if (!c->mlp) c->mlp = new Mlp();
    if (c->mlp->cap < m) SCUDA(mlp_alloc(*c->mlp, std::max(m, 1024)));
  }
  if ((rc = ensure_scratch(c, std::max(m, 2 * k)))) return rc;  // records and partials of 2k request slots

  // initial live set and its likelihoods (with the per-detector sums)
  SCUDA(cudaSetDevice(c->device));
  k_init_live<<<(m + 127) / 128, 128, 0, c->stream>>>(S, st->P.live_u, st->init_theta);
  SCUDA(cudaGetLastError());
  {
    cudaError_t e = cudaMemsetAsync(st->P.live_vv, 0, sizeof(double) * m * SWIG_MAX_DET, c->stream);
    if (e != cudaSuccess) {
    } else if (het) {
      e = launch_loglike_het(L, c->B, st->init_theta, m, st->P.live_logl, c->stream, st->P.live_kap, st->P.live_vv);
    } else {
      e = mixed ? launch_loglike_mixed(L, c->B, st->init_theta, m, st->P.live_logl, c->stream, st->P.live_kap)
                : launch_loglike_fp64(L, c->B, st->init_theta, m, st->P.live_logl, c->stream, st->P.live_kap);
    }
    SCUDA(e);
  }
  NSGlobal g0;
  std::memset(&g0, 0, sizeof(g0));
  g0.logx = 0.0;
  g0.logz = -INFINITY;
  g0.chains_done = k;
  g0.status = ST_RUNNING;
  SCUDA(cudaMemcpyAsync(st->P.g, &g0, sizeof(g0), cudaMemcpyHostToDevice, c->stream));
  SCUDA(cudaMemsetAsync(st->P.pending, 0, sizeof(int) * k, c->stream));
  SCUDA(cudaMemsetAsync(st->P.req, 0, sizeof(int) * 2 * k, c->stream));
  SCUDA(cudaMemsetAsync(st->P.done_cnt, 0, sizeof(int) * 2 * k, c->stream));
  SCUDA(cudaMemsetAsync(st->P.chains, 0, sizeof(ChainState) * k, c->stream));
  c->n_launches += het ? 3 : (mixed ? 5 : 4);  // init draw + batched likelihood

  R.kern = het ? pick_het_kernel(L.n_det) : pick_kernel(L.n_det, mixed);
  R.threads = het ? kHetThreads : kFlowThreads;
  if (R.learned) SCUDA(mlp_init(*c->mlp, c->cfg.seed ^ 0x4D4C5050ull, c->stream, &c->n_launches));
  R.du.clear();
  R.dl.clear();
  R.dw.clear();
  R.total_iters = 0;
  R.finished = false;
  return SWIG_OK;
}

// Reset the per-launch counters of the NS state before a launch.
int run_reset(swig_ctx* c, RunState& R) {
  NSGlobal gl;
  SCUDA(cudaMemcpyAsync(&gl, R.st->P.g, sizeof(gl), cudaMemcpyDeviceToHost, c->stream));
  SCUDA(cudaStreamSynchronize(c->stream));
  gl.iters_launch = 0;
  gl.n_dead = 0;
  gl.status = ST_RUNNING;
  gl.error = 0;
  gl.bar_count = 0;
  SCUDA(cudaMemcpyAsync(R.st->P.g, &gl, sizeof(gl), cudaMemcpyHostToDevice, c->stream));
  return SWIG_OK;
}

// After a launch: the NS state, its dead points, and whether the run is over.
int run_collect(swig_ctx* c, RunState& R) {
  SCUDA(cudaMemcpyAsync(&R.gh, R.st->P.g, sizeof(R.gh), cudaMemcpyDeviceToHost, c->stream));
  SCUDA(cudaStreamSynchronize(c->stream));
  const NSGlobal& gh = R.gh;
  if (gh.error) return fail(c, gh.error, gh.error == SWIG_E_TIMEOUT ? "a bounded device wait expired" : "device error");
  c->d2h_bytes += sizeof(gh);
  const int nd = R.nd;
  if (gh.n_dead > 0) {
    c->d2h_bytes += (size_t)gh.n_dead * (nd + 2) * sizeof(double);
    const size_t n0 = R.dl.size();
    R.du.resize((n0 + gh.n_dead) * nd);
    R.dl.resize(n0 + gh.n_dead);
    R.dw.resize(n0 + gh.n_dead);
    SCUDA(cudaMemcpy(R.du.data() + n0 * nd, R.st->P.dead_u, sizeof(double) * gh.n_dead * nd, cudaMemcpyDeviceToHost));
    SCUDA(cudaMemcpy(R.dl.data() + n0, R.st->P.dead_logl, sizeof(double) * gh.n_dead, cudaMemcpyDeviceToHost));
    SCUDA(cudaMemcpy(R.dw.data() + n0, R.st->P.dead_logw, sizeof(double) * gh.n_dead, cudaMemcpyDeviceToHost));
  }
  R.total_iters = gh.iter;
  R.finished = gh.status == ST_TERMINATED || R.total_iters >= c->cfg.max_iter;
  return SWIG_OK;
}

// Final live points, the samples' parameters (and post-hoc distances), the
// result and the profile counters.
int run_finish(swig_ctx* c, RunState& R, swig_result* out) {
  const int m = R.m, k = R.k, nd = R.nd;
  const bool mixed = R.mixed, het = R.het;
  const LikeConst& L = c->L;
  const SamplerConst& S = R.S;
  SamplerState* st = R.st;
  const NSGlobal& gh = R.gh;
  std::vector<double>& du = R.du;
  std::vector<double>& dl = R.dl;
  std::vector<double>& dw = R.dw;
  // final live points, X/m each
  std::vector<double> lu((size_t)m * nd), ll(m);
  SCUDA(cudaMemcpy(lu.data(), st->P.live_u, sizeof(double) * lu.size(), cudaMemcpyDeviceToHost));
  SCUDA(cudaMemcpy(ll.data(), st->P.live_logl, sizeof(double) * m, cudaMemcpyDeviceToHost));
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ll[a] < ll[b]; });
  double logz = gh.logz;
  for (int i : order) {
    const double w = ll[i] + gh.logx - std::log((double)m);
    du.insert(du.end(), lu.begin() + (size_t)i * nd, lu.begin() + (size_t)(i + 1) * nd);
    dl.push_back(ll[i]);
    dw.push_back(w);
    const double hi = std::max(logz, w);
    logz = std::isfinite(hi) ? hi + std::log(std::exp(logz - hi) + std::exp(w - hi)) : hi;
  }
  const size_t n_dead = dl.size();
  double info = 0.0, sum_p2 = 0.0;
  for (size_t i = 0; i < n_dead; ++i) {
    const double p = std::exp(dw[i] - logz);
    info += p * (dl[i] - logz);
    sum_p2 += p * p;
  }
  // counters
  std::vector<ChainState> ch(k);
  SCUDA(cudaMemcpy(ch.data(), st->P.chains, sizeof(ChainState) * k, cudaMemcpyDeviceToHost));
  // theta of every dead point via the device prior transform
  c->out_theta.assign(n_dead * SWIG_N_PARAMS, 0.0);
  {
    double *du_d = nullptr, *th_d = nullptr;
    SCUDA(cudaMalloc(&du_d, sizeof(double) * std::max<size_t>(1, du.size())));
    SCUDA(cudaMalloc(&th_d, sizeof(double) * std::max<size_t>(1, c->out_theta.size())));
    SCUDA(cudaMemcpy(du_d, du.data(), sizeof(double) * du.size(), cudaMemcpyHostToDevice));
    k_dead_theta<<<(unsigned)((n_dead + 127) / 128), 128, 0, c->stream>>>(S, du_d, (int)n_dead, th_d);
    ++c->n_launches;
    if (L.dist_marg) {
      // post-hoc distances: the kappa sums of every sample, then a draw from
      // its conditional distance posterior
      const int chunk = 4096;
      double *kap_d = nullptr, *ll_d = nullptr;
      cudaError_t e = cudaMalloc(&kap_d, sizeof(double) * 2 * SWIG_MAX_DET * chunk);
      if (e == cudaSuccess) e = cudaMalloc(&ll_d, sizeof(double) * chunk);
      for (size_t off = 0; e == cudaSuccess && off < n_dead; off += chunk) {
        const int mm = (int)std::min<size_t>(chunk, n_dead - off);
        if (ensure_scratch(c, mm)) {
          e = cudaErrorMemoryAllocation;
          break;
        }
        e = mixed ? launch_loglike_mixed(L, c->B, th_d + off * SWIG_N_PARAMS, mm, ll_d, c->stream, kap_d)
                  : launch_loglike_fp64(L, c->B, th_d + off * SWIG_N_PARAMS, mm, ll_d, c->stream, kap_d);
        if (e == cudaSuccess)
          e = launch_distance_draw(L, c->B, kap_d, mm, (long long)off, S.key0, S.key1, th_d + off * SWIG_N_PARAMS,
                                   c->stream);
        c->n_launches += mixed ? 5 : 4;
      }
      if (kap_d) cudaFree(kap_d);
      if (ll_d) cudaFree(ll_d);
      if (e != cudaSuccess) {
        cudaFree(du_d);
        cudaFree(th_d);
        SCUDA(e);
      }
    }
    if (L.tm_n > 0) {
      // post-hoc t_c: the node log weights of every sample, then a draw from
      // its conditional on the time grid
      const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(4096, ((int64_t)1 << 26) / L.tm_n));
      double* ll_d = nullptr;
      float* ell_d = nullptr;
      cudaError_t e = cudaMalloc(&ll_d, sizeof(double) * chunk);
      if (e == cudaSuccess) e = cudaMalloc(&ell_d, sizeof(float) * (size_t)chunk * L.tm_n);
      for (size_t off = 0; e == cudaSuccess && off < n_dead; off += chunk) {
        const int mm = (int)std::min<size_t>(chunk, n_dead - off);
        if (ensure_scratch(c, mm)) {
          e = cudaErrorMemoryAllocation;
          break;
        }
        e = launch_loglike_het(L, c->B, th_d + off * SWIG_N_PARAMS, mm, ll_d, c->stream, nullptr, nullptr, ell_d);
        if (e == cudaSuccess)
          e = launch_time_draw(L, c->B, ell_d, mm, (long long)off, S.key0, S.key1, th_d + off * SWIG_N_PARAMS,
                               c->stream);
        c->n_launches += 3;
      }
      if (ll_d) cudaFree(ll_d);
      if (ell_d) cudaFree(ell_d);
      if (e != cudaSuccess) {
        cudaFree(du_d);
        cudaFree(th_d);
        SCUDA(e);
      }
    }
    c->h2d_bytes += sizeof(double) * du.size();
    c->d2h_bytes += sizeof(double) * c->out_theta.size();
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(c->out_theta.data(), th_d, sizeof(double) * c->out_theta.size(), cudaMemcpyDeviceToHost);
    cudaFree(du_d);
    cudaFree(th_d);
    SCUDA(e);
  }
  c->out_logl = dl;
  c->out_logw.resize(n_dead);
  for (size_t i = 0; i < n_dead; ++i) c->out_logw[i] = dw[i];
  // normalise so that logsumexp(logw) = log Z (already the case by construction)
  out->logz = logz;
  out->info = info;
  out->logz_err = std::sqrt(std::max(info, 0.0) / m);
  out->ess = sum_p2 > 0 ? 1.0 / sum_p2 : 0.0;
  out->n_dead = (int64_t)n_dead;
  out->n_iter = R.total_iters;
  // evaluations: the initial m plus the chains' counters accumulated on device
  long long ne = m, nf = m;
  for (const ChainState& q : ch) {
    ne += q.n_evals;
    nf += q.n_full;
  }
  out->n_evals = ne;
  out->n_sweep_evals = nf;
  out->status = gh.status == ST_TERMINATED ? 0 : 1;
  out->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - R.t_start).count();
  c->last = *out;
  c->profile[0] = (double)gh.rounds;
  c->profile[1] = gh.t_bound * 1e-9;
  c->profile[2] = gh.t_ctrl * 1e-9;
  c->profile[3] = gh.t_wait_ctrl * 1e-9;
  c->profile[4] = gh.t_sweep * 1e-9;
  c->profile[5] = gh.t_wait_sweep * 1e-9;
  c->profile[6] = R.persistent_ms;
  c->profile[7] = (double)R.persistent_launches;
  c->profile[8] = (double)c->n_launches;
  c->profile[9] = (double)c->h2d_bytes;
  c->profile[10] = (double)c->d2h_bytes;
  // bin-detector evaluations (heterodyned: bins of the coarse grid)
  c->profile[11] = (double)nf * (double)L.n_det * (double)(het ? c->B.het_nb : L.n_bins);
  c->profile[12] = (double)gh.c_result;
  c->profile[13] = (double)gh.c_step;
  c->profile[14] = (double)gh.c_prop;
  c->profile[15] = (double)gh.c_free;
  c->profile[16] = (double)gh.c_setup;
  c->profile[17] = (double)gh.n_free;
  c->profile[18] = (double)gh.n_setup;
  c->profile[19] = (double)gh.n_step;
  c->profile[20] = R.learn_ms;
  c->profile[21] = (double)R.learn_rounds;
  c->profile[22] = (double)gh.f_units;
  c->profile[23] = (double)gh.f_unit_cyc;
  c->profile[24] = (double)gh.f_idle_cyc;
  {
    std::vector<unsigned long long> cp(4 * (size_t)S.n_ctas);
    SCUDA(cudaMemcpy(cp.data(), st->cta_prof, sizeof(unsigned long long) * cp.size(), cudaMemcpyDeviceToHost));
    c->cta_profile.assign(cp.begin(), cp.end());
  }
  return SWIG_OK;
}

// The persistent launches of one run until termination or the iteration cap.
int run_loop_single(swig_ctx* c, RunState& R) {
  int rc = SWIG_OK;
  SCUDA(cudaFuncSetAttribute(R.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R.smem));
  int per_sm = 0;
  SCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, R.kern, R.threads, R.smem));
  if (per_sm < 1 || R.S.n_ctas > per_sm * c->sm_count)
    return fail(c, SWIG_E_CUDA, "persistent kernel cannot be co-resident on this device");
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  SCUDA(cudaEventCreate(&ev0));
  SCUDA(cudaEventCreate(&ev1));
  while (!R.finished) {
    if ((rc = run_reset(c, R))) break;
    if (R.learned) {
      // retrain on the current live set, then freeze the output rows of
      // this snapshot for the launch's iterations
      Mlp& N = *c->mlp;
      cudaError_t e = cudaEventRecord(ev0, c->stream);
      if (e == cudaSuccess) e = mlp_targets(N, R.st->P.live_u, R.m, R.nd, 2 * R.nd, c->stream, &c->n_launches);
      if (e == cudaSuccess)
        e = mlp_train(N, R.m, R.nd, R.learn_rounds == 0 ? 4 * R.learn_steps : R.learn_steps, R.learn_lr, c->stream,
                      &c->n_launches);
      if (e == cudaSuccess) e = mlp_forward(N, R.m, c->stream, &c->n_launches);
      if (e == cudaSuccess) e = cudaEventRecord(ev1, c->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
      if (e != cudaSuccess) {
        rc = fail(c, SWIG_E_CUDA, std::string("learned proposal training: ") + cudaGetErrorString(e));
        break;
      }
      R.learn_ms += ms;
      ++R.learn_rounds;
      R.st->P.learn_out = N.out;
    }
    void* args[] = {(void*)&c->L, (void*)&R.S, (void*)&c->B, (void*)&R.st->P};
    cudaError_t e = cudaEventRecord(ev0, c->stream);
    if (e == cudaSuccess)
      e = cudaLaunchCooperativeKernel(R.kern, dim3(R.S.n_ctas), dim3(R.threads), args, R.smem, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    if (e != cudaSuccess) {
      rc = fail(c, SWIG_E_CUDA, std::string("persistent launch: ") + cudaGetErrorString(e));
      break;
    }
    R.persistent_ms += ms;
    ++R.persistent_launches;
    ++c->n_launches;
    if ((rc = run_collect(c, R))) break;
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  return rc;
}

// Events of one campaign that can share a launch: full grid, mixed precision,
// covariance proposal, the same detector count, chains per event and device.
bool batchable(swig_ctx* const* ctxs, const std::vector<RunState>& R, int i0, int i1) {
  for (int i = i0; i < i1; ++i) {
    if (R[i].het || !R[i].mixed || R[i].learned) return false;
    if (ctxs[i]->L.n_det != ctxs[i0]->L.n_det || R[i].k != R[i0].k || ctxs[i]->device != ctxs[i0]->device) return false;
  }
  return true;
}

// One group of events in k_ns_multi launches until every one is finished.
int run_loop_multi(swig_ctx* const* ctxs, std::vector<RunState>& R, int i0, int i1) {
  swig_ctx* c0 = ctxs[i0];
  const int n_det = c0->L.n_det, k = R[i0].k;
  // shared-memory layout: every event's slice data, then the per-warp records
  // or the boundary's sort buffers
  std::vector<int> off(i1 - i0);
  size_t fixed = 0, tail = 0;
  int grid = 1;
  for (int i = i0; i < i1; ++i) {
    off[i - i0] = (int)fixed;
    fixed += R[i].fixed;
    tail = std::max(tail, R[i].tail);
    grid = std::max(grid, ctxs[i]->L.n_slices);
  }
  // after the data and the records / sort buffers: each control warp's slots
  // for the chains it serves (warp-parallel control)
  const int n_ctrl = std::max(1, std::min(4, ((i1 - i0) * k + grid - 1) / grid));
  const int ctl_slots = ((i1 - i0) * k + grid * n_ctrl - 1) / (grid * n_ctrl);
  const size_t ctl_off = (fixed + tail + 15) & ~(size_t)15;
  const size_t smem = ctl_off + (size_t)n_ctrl * ctl_slots * (sizeof(ChainState) + sizeof(EvalRecord));
  void* kern = pick_multi_kernel(n_det);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFlowThreads, smem);
  if (e != cudaSuccess) return fail(c0, SWIG_E_CUDA, std::string("multi-event kernel set-up: ") + cudaGetErrorString(e));
  if (per_sm < 1 || grid > per_sm * c0->sm_count)
    return fail(c0, SWIG_E_CUDA, "multi-event persistent kernel cannot be co-resident on this device");
  NSGlobal* gb = nullptr;
  EventDesc* evd = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int rc = SWIG_OK;
  e = cudaMalloc(&gb, sizeof(NSGlobal));
  if (e == cudaSuccess) e = cudaMalloc(&evd, sizeof(EventDesc) * (i1 - i0));
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  std::vector<EventDesc> hd;
  std::vector<int> idx;
  while (e == cudaSuccess && rc == SWIG_OK) {
    hd.clear();
    idx.clear();
    for (int i = i0; i < i1; ++i) {
      if (R[i].finished) continue;
      if ((rc = run_reset(ctxs[i], R[i]))) break;
      EventDesc d;
      d.L = ctxs[i]->L;
      d.S = R[i].S;
      d.S.par_out = 0;  // the campaign kernel steps out one end at a time (same evaluations and results)
      d.S.n_slots = d.S.nrep;
      d.B = ctxs[i]->B;
      d.P = R[i].st->P;
      d.smem_off = off[i - i0];
      hd.push_back(d);
      idx.push_back(i);
    }
    if (rc || hd.empty()) break;
    for (int i : idx) {
      e = cudaStreamSynchronize(ctxs[i]->stream);
      if (e != cudaSuccess) break;
    }
    NSGlobal g0;
    std::memset(&g0, 0, sizeof(g0));
    if (e == cudaSuccess) e = cudaMemcpy(gb, &g0, sizeof(g0), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(evd, hd.data(), sizeof(EventDesc) * hd.size(), cudaMemcpyHostToDevice);
    int n_ev = (int)hd.size();
    int n_ctrl_arg = n_ctrl;
    int dyn_off = (int)fixed, ctl_off_arg = (int)ctl_off, ctl_slots_arg = ctl_slots;
    void* args[] = {(void*)&evd,    (void*)&n_ev,        (void*)&gb,           (void*)&n_ctrl_arg,
                    (void*)&dyn_off, (void*)&ctl_off_arg, (void*)&ctl_slots_arg};
    if (e == cudaSuccess) e = cudaEventRecord(ev0, c0->stream);
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kFlowThreads), args, smem, c0->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev1, c0->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    NSGlobal gh;
    if (e == cudaSuccess) e = cudaMemcpy(&gh, gb, sizeof(gh), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    if (gh.error) {
      rc = fail(c0, gh.error, gh.error == SWIG_E_TIMEOUT ? "a bounded device wait expired" : "device error");
      break;
    }
    for (int i : idx) {
      R[i].persistent_ms += ms;  // the launch's wall time, shared by its events
      ++R[i].persistent_launches;
      if ((rc = run_collect(ctxs[i], R[i]))) break;
    }
    ++c0->n_launches;
  }
  if (e != cudaSuccess && rc == SWIG_OK)
    rc = fail(c0, SWIG_E_CUDA, std::string("multi-event launch: ") + cudaGetErrorString(e));
  if (gb) cudaFree(gb);
  if (evd) cudaFree(evd);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  return rc;
}

}  // namespace

extern "C" {

int swig_autotune(swig_ctx* c, int iters, double* out, int n) {
  if (!c) return SWIG_E_ARG;
  if (iters < 1) return fail(c, SWIG_E_ARG, "autotune needs at least one iteration");
  if (out && n > 0) out[0] = 0.0;
  const swig_sampler_cfg saved = c->cfg;
  if (!c->cfg_set) return fail(c, SWIG_E_STATE, "sampler settings not set");
  if (saved.likelihood != SWIG_LIKE_FULL || saved.precision != SWIG_PREC_MIXED ||
      saved.proposal != SWIG_PROPOSAL_COV)
    return SWIG_OK;
  const int cand[4][2] = {{1, 0}, {1, 1}, {2, 0}, {3, 0}};
  double rate[4] = {0.0, 0.0, 0.0, 0.0};
  int best = 0;
  for (int i = 0; i < 4; ++i) {
    c->cfg = saved;
    c->cfg.flow_parts = cand[i][0];
    c->cfg.stepout_one_end = cand[i][1];
    c->cfg.max_iter = iters;
    swig_result r;
    const int rc = swig_run(c, &r);
    if (rc != SWIG_OK) {
      c->cfg = saved;
      return rc;
    }
    rate[i] = c->profile[6] > 0.0 ? (double)r.n_sweep_evals / (c->profile[6] * 1e-3) : 0.0;
    if (rate[i] > rate[best]) best = i;
  }
  c->cfg = saved;
  c->cfg.flow_parts = cand[best][0];
  c->cfg.stepout_one_end = cand[best][1];
  if (out && n > 0) {
    out[0] = 4.0;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 3; ++j)
        if (1 + 3 * i + j < n) out[1 + 3 * i + j] = j == 0 ? cand[i][0] : j == 1 ? cand[i][1] : rate[i];
  }
  return SWIG_OK;
}

int swig_run(swig_ctx* c, swig_result* out) {
  if (!c) return SWIG_E_ARG;
  if (!out) return fail(c, SWIG_E_ARG, "null result pointer");
  std::memset(out, 0, sizeof(*out));
  RunState R;
  int rc = run_setup(c, R);
  if (!rc) rc = run_loop_single(c, R);
  if (rc) return rc;
  return run_finish(c, R, out);
}

int swig_run_batch(swig_ctx** ctxs, int n_ctx, swig_result* outs) {
  if (!ctxs || !outs || n_ctx < 1) return SWIG_E_ARG;
  for (int i = 0; i < n_ctx; ++i) {
    if (!ctxs[i]) return SWIG_E_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(ctxs[i], SWIG_E_ARG, "a context appears twice in the batch");
    std::memset(&outs[i], 0, sizeof(outs[i]));
  }
  std::vector<RunState> R(n_ctx);
  for (int i = 0; i < n_ctx; ++i) {
    const int rc = run_setup(ctxs[i], R[i]);
    if (rc) return rc;
  }
  // Events share a launch in groups of similar grid size: the events of a
  // launch advance their NS iterations in step, so a short event grouped with
  // a long one would wait for it.  Greedy groups over the events sorted by
  // grid size: at most kMaxEvents, within 1.5x of the group's smallest grid,
  // their chains within kMaxChains, their slices within one CTA's shared
  // memory.
  std::vector<int> order(n_ctx);
  for (int i = 0; i < n_ctx; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ctxs[a]->L.n_bins < ctxs[b]->L.n_bins; });
  std::vector<swig_ctx*> oc(n_ctx);
  std::vector<RunState> orr(n_ctx);
  for (int i = 0; i < n_ctx; ++i) {
    oc[i] = ctxs[order[i]];
    orr[i] = R[order[i]];
  }
  int i0 = 0;
  while (i0 < n_ctx) {
    int i1 = i0 + 1;
    if (batchable(oc.data(), orr, i0, i0 + 1)) {
      size_t fixed = orr[i0].fixed, tail = orr[i0].tail;
      while (i1 < n_ctx && i1 - i0 < kMaxEvents && batchable(oc.data(), orr, i0, i1 + 1) &&
             (i1 + 1 - i0) * orr[i0].k <= kMaxChains && oc[i1]->L.n_bins <= 1.5 * oc[i0]->L.n_bins &&
             fixed + orr[i1].fixed + std::max(tail, orr[i1].tail) <= 212 * 1024) {
        fixed += orr[i1].fixed;
        tail = std::max(tail, orr[i1].tail);
        ++i1;
      }
    }
    int rc = i1 - i0 == 1 ? run_loop_single(oc[i0], orr[i0]) : run_loop_multi(oc.data(), orr, i0, i1);
    if (rc) return rc;
    for (int i = i0; i < i1; ++i)
      if ((rc = run_finish(oc[i], orr[i], &outs[order[i]]))) return rc;
    i0 = i1;
  }
  return SWIG_OK;
}

int swig_get_profile(swig_ctx* c, double* out, int n) {
  if (!c) return SWIG_E_ARG;
  if (!out || n < 0) return fail(c, SWIG_E_ARG, "null output");
  for (int i = 0; i < n && i < 25; ++i) out[i] = c->profile[i];
  for (int i = 25; i < n && i - 25 < (int)c->cta_profile.size(); ++i) out[i] = c->cta_profile[i - 25];
  return SWIG_OK;
}

int swig_get_samples(swig_ctx* c, double* theta, double* logl, double* logw, int64_t cap, int64_t* n_out) {
  if (!c) return SWIG_E_ARG;
  if (!n_out) return fail(c, SWIG_E_ARG, "null n_out");
  const int64_t n = (int64_t)c->out_logl.size();
  *n_out = n;
  if (cap == 0) return SWIG_OK;
  if (cap < n || !theta || !logl || !logw) return fail(c, SWIG_E_ARG, "capacity below the number of samples or null buffer");
  std::memcpy(theta, c->out_theta.data(), sizeof(double) * n * SWIG_N_PARAMS);
  std::memcpy(logl, c->out_logl.data(), sizeof(double) * n);
  std::memcpy(logw, c->out_logw.data(), sizeof(double) * n);
  return SWIG_OK;
}

}  // extern "C"
