// Heterodyned (relative-binning) likelihood (Sec. 3.4 of the paper) on the device.
//
// With the fiducial waveform h0 the ratio r_i(f) = h_i(f) / h0_i(f) is, for
// this model, (C_i / C0_i) exp(-2 pi i (dP(f) + f dtau_i)) with dP = P - P0 and
// dtau_i = tau_i - tau0_i (the f^-7/6 amplitude cancels).  It is evaluated at
// the N_b + 1 bin edges and taken linear inside each bin:
//   r0_b = (r(e_b) + r(e_b+1)) / 2,  r1_b = (r(e_b+1) - r(e_b)) / (e_b+1 - e_b),
//   Z_i  = sum_b A0_ib r0_b + A1_ib r1_b,
//   HH_i = sum_b B0_ib |r0_b|^2 + 2 B1_ib Re(r0_b conj(r1_b)),
// with the summary data A0, A1, B0, B1 (host FP64, stored FP32).  dP at an
// edge is a double-float sum of (c_j - c0_j) phi_j(f_e) (it can reach hundreds
// of cycles far from the fiducial); the contraction itself is FP32 per bin with
// a pairwise (warp-shuffle) reduction and an FP64 epilogue.
//
// Time marginalisation (t_c marginalised, Sec. 3.1 and App. A).  Z_i is
// linear in the edge values, Z_i = sum_e g_ie r_i(e) with hat-function weights
// g_ie = (A0_ib/2 - A1_ib/w_b) from the bin above the edge plus
// (A0_ib/2 + A1_ib/w_b) from the bin below.  A common geocentric shift dt
// multiplies r_i(e) by exp(-2 pi i f_e dt) in every detector, so the network
// overlap at a grid node is one sum over edges,
//   Z(dt_j) = sum_e y_e exp(-2 pi i f_e dt_j),   y_e = sum_i g_ie r_i(e),
// with the templates built at the fiducial's t_c.  <h|h> is the same at every
// node (a time shift only rotates h) and is taken there once.
#pragma once

#include "device_common.cuh"

namespace swig {

struct HetTables {
  int n_bins;                 // N_b
  const float* edge_basis;    // [2 * NBASIS][N_b + 1] phi_j(f_e): row 2j hi parts, row 2j+1 lo parts
  const float* edge_f;        // [2][N_b + 1] f_e: hi parts, lo parts
  const float* inv_width;     // [N_b] 1 / (e_{b+1} - e_b)
  const float4* coef;         // [n_det][N_b] (A0.re, A0.im, A1.re, A1.im)
  const float2* coefB;        // [n_det][N_b] (B0, B1)
  const EvalRecord* fid;      // fiducial record
  const float2* tm_g;         // [n_det][N_b + 1] time marginalisation: edge weights g_ie
  const float2* tm_w;         // [N_b + 1] exp(-2 pi i f_e dt), one grid step
  // non-uniform FFT form of the time pass (see het_nufft_tables)
  const float* nu_wt;
  const float* nu_corr;
  const float2* nu_tw;
  const int4* nu_piece;  // gather pieces (first entry, entries, first edge)
  const int4* nu_point;  // grid points with entries (point, first piece, pieces)
  // chunk anchors (kernels.h HetChunkRow)
  int n_chunks;
  const float* chunk;  // [HC_ROWS][n_chunks]
  const float* dfe;    // [n_chunks][32]
};

__host__ __device__ inline HetTables het_tables(const DeviceBuffers& B) {
  HetTables H;
  H.n_bins = B.het_nb;
  H.edge_basis = B.het_edge_basis;
  H.edge_f = B.het_edge_f;
  H.inv_width = B.het_inv_width;
  H.coef = B.het_coef;
  H.coefB = B.het_coefB;
  H.fid = B.het_fid;
  H.tm_g = B.het_tm_g;
  H.tm_w = B.het_tm_w;
  H.nu_wt = B.het_nu_wt;
  H.nu_corr = B.het_nu_corr;
  H.nu_tw = B.het_nu_tw;
  H.nu_piece = B.het_nu_piece;
  H.nu_point = B.het_nu_point;
  H.n_chunks = B.het_nc;
  H.chunk = B.het_chunk;
  H.dfe = B.het_dfe;
  return H;
}

// Per-evaluation constants: coefficient and delay differences from the
// fiducial in double-float, and rho_i = C_i / C0_i.
template <int NDET>
struct HetPrep {
  dfl dc[NBASIS];
  dfl dtau[NDET];
  float rho_re[NDET], rho_im[NDET];
};

template <int NDET>
__device__ inline void het_prepare(const LikeConst& L, const HetTables& H, const EvalRecord& r, HetPrep<NDET>& p) {
  const EvalRecord& f0 = *H.fid;
#pragma unroll
  for (int j = 0; j < NBASIS; ++j) p.dc[j] = df_from_double(r.c[j] - f0.c[j]);
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
    p.dtau[i] = df_from_double(r.tau[i] - f0.tau[i]);
    const double iden = L.het_fid_iden[i];
    p.rho_re[i] = (float)((r.cre[i] * f0.cre[i] + r.cim[i] * f0.cim[i]) * iden);
    p.rho_im[i] = (float)((r.cim[i] * f0.cre[i] - r.cre[i] * f0.cim[i]) * iden);
  }
}

// Anchor of chunk q for one evaluation (one thread per chunk; rows of the
// chunk table are read coalesced across threads): the phase difference
// dP(f) = sum_j (c_j - c0_j) phi_j(f) at the chunk's first edge f_a in
// double-float, its scaled derivatives a_1 (double-float sum, stored FP32)
// and a_2..a_10 (FP32), per detector frac(dP(f_a) + f_a dtau_i), and whether
// this evaluation's Taylor remainder bound sum_j |c_j - c0_j| HC_BND_j
// exceeds kHetTaylorEps (then the chunk is taken edge by edge).
template <int NDET>
__device__ inline void het_anchor(const HetTables& H, const HetPrep<NDET>& p, int q, float* out) {
  const int nc = H.n_chunks;
  const float* T = H.chunk + q;
  auto row = [&](int r) { return __ldg(T + (size_t)r * nc); };
  dfl A = {0.0f, 0.0f}, S = {0.0f, 0.0f};
  float a[kHetPoly], R = 0.0f;
#pragma unroll
  for (int n = 0; n < kHetPoly; ++n) a[n] = 0.0f;
#pragma unroll
  for (int j = 0; j < NBASIS; ++j) {
    const dfl c = p.dc[j];
    R = fmaf(fabsf(c.hi), row(HC_BND + j), R);
    A = df_add(A, df_mul(c, dfl{row(HC_VAL_HI + j), row(HC_VAL_LO + j)}));
    S = df_add(S, df_mul(c, dfl{row(HC_D1_HI + j), row(HC_D1_LO + j)}));
#pragma unroll
    for (int n = 0; n < kHetPoly; ++n) a[n] = fmaf(c.hi, row(HC_POLY + n * NBASIS + j), a[n]);
  }
  out[0] = S.hi + S.lo;
#pragma unroll
  for (int n = 0; n < kHetPoly; ++n) out[1 + n] = a[n];
  const dfl fa = {row(HC_FA_HI), row(HC_FA_LO)};
#pragma unroll
  for (int i = 0; i < NDET; ++i) out[kHetAncPhase + i] = df_frac(df_add(A, df_mul(fa, p.dtau[i])));
  out[kHetAncInvS] = row(HC_INV_S);
  out[kHetAncExact] = R > kHetTaylorEps ? 1.0f : 0.0f;
}

// Bins [base, base + 31) of the contraction, accumulated into the lane's
// per-detector sums: lane l holds edge base + l, bin base + l uses edges l and
// l + 1 (the next edge by a shuffle).  All 32 lanes must call it together.
// With TM the lanes also store the network edge products y_e of the time
// marginalisation (each edge once: lanes 0..30, and the last edge).
template <int NDET, bool TM = false>
__device__ inline void het_chunk(const HetTables& H, const HetPrep<NDET>& p, int base, int lane, float* zr, float* zi,
                                 float* hh, float2* y = nullptr) {
  const float twopi = 6.283185307179586f;
  const int e = base + lane;
  float er[NDET], ei[NDET];
  if (e <= H.n_bins) {
    const size_t ne = (size_t)H.n_bins + 1;  // edges; lanes read consecutive edges of each row
    dfl dp = {0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < NBASIS; ++j)
      dp = df_add(dp, df_mul(p.dc[j], dfl{H.edge_basis[2 * j * ne + e], H.edge_basis[(2 * j + 1) * ne + e]}));
    const dfl fe = {H.edge_f[e], H.edge_f[ne + e]};
#pragma unroll
    for (int i = 0; i < NDET; ++i) {
      const float ph = df_frac(df_add(dp, df_mul(fe, p.dtau[i])));
      float s, co;
      __sincosf(twopi * ph, &s, &co);  // exp(-2 pi i ph) = co - i s
      er[i] = p.rho_re[i] * co + p.rho_im[i] * s;
      ei[i] = p.rho_im[i] * co - p.rho_re[i] * s;
    }
    if (TM && (lane < 31 || e == H.n_bins)) {
      float yr = 0.0f, yi = 0.0f;
#pragma unroll
      for (int i = 0; i < NDET; ++i) {
        const float2 g = H.tm_g[(size_t)i * ne + e];
        yr += g.x * er[i] - g.y * ei[i];
        yi += g.x * ei[i] + g.y * er[i];
      }
      y[e] = make_float2(yr, yi);
    }
  } else {
#pragma unroll
    for (int i = 0; i < NDET; ++i) er[i] = ei[i] = 0.0f;
  }
  const int b = base + lane;
  const bool has_bin = lane < 31 && b < H.n_bins;
  const float iw = has_bin ? H.inv_width[b] : 0.0f;
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
    const float nr = __shfl_down_sync(0xffffffffu, er[i], 1);
    const float ni = __shfl_down_sync(0xffffffffu, ei[i], 1);
    if (has_bin) {
      const float r0r = 0.5f * (er[i] + nr), r0i = 0.5f * (ei[i] + ni);
      const float r1r = (nr - er[i]) * iw, r1i = (ni - ei[i]) * iw;
      const float4 a = H.coef[(size_t)i * H.n_bins + b];
      const float2 bb = H.coefB[(size_t)i * H.n_bins + b];
      zr[i] += a.x * r0r - a.y * r0i + a.z * r1r - a.w * r1i;
      zi[i] += a.x * r0i + a.y * r0r + a.z * r1i + a.w * r1r;
      hh[i] += bb.x * (r0r * r0r + r0i * r0i) + 2.0f * bb.y * (r0r * r1r + r0i * r1i);
    }
  }
}

// Per-lane table data of one chunk step: edge offset, bin width and summary
// data of the lane's bin.
template <int NDET>
struct HetBinData {
  float d, iw;
  float4 a[NDET];
  float2 bb[NDET];
};

// het_chunk with the phase from chunk q's anchor `anc` (het_anchor) and the
// lane's table data t (het_read_stage): lane l holds edge 31 q + l at
// x = (f_e - f_a) / S, dP = sum_n a_n x^n (degree 10, FP32 Horner),
// phase_i = frac(anchor_i + dP + (f_e - f_a) dtau_i).
template <int NDET, bool TM = false>
__device__ inline void het_chunk_anc(const HetTables& H, const HetPrep<NDET>& p, const float* anc, int q, int lane,
                                     const HetBinData<NDET>& t, float* zr, float* zi, float* hh,
                                     float2* y = nullptr) {
  const float twopi = 6.283185307179586f;
  const int base = 31 * q, e = base + lane;
  float er[NDET], ei[NDET];
  if (e <= H.n_bins) {
    const float x = t.d * anc[kHetAncInvS];
    float v = anc[kHetPoly];
#pragma unroll
    for (int n = kHetPoly - 1; n >= 0; --n) v = fmaf(v, x, anc[n]);
    v *= x;
#pragma unroll
    for (int i = 0; i < NDET; ++i) {
      float ph = anc[kHetAncPhase + i] + fmaf(t.d, p.dtau[i].hi, v);
      ph -= round_nearest(ph);
      float s, co;
      __sincosf(twopi * ph, &s, &co);  // exp(-2 pi i ph) = co - i s
      er[i] = p.rho_re[i] * co + p.rho_im[i] * s;
      ei[i] = p.rho_im[i] * co - p.rho_re[i] * s;
    }
    if (TM && (lane < 31 || e == H.n_bins)) {
      float yr = 0.0f, yi = 0.0f;
      const size_t ne = (size_t)H.n_bins + 1;
#pragma unroll
      for (int i = 0; i < NDET; ++i) {
        const float2 g = H.tm_g[(size_t)i * ne + e];
        yr += g.x * er[i] - g.y * ei[i];
        yi += g.x * ei[i] + g.y * er[i];
      }
      y[e] = make_float2(yr, yi);
    }
  } else {
#pragma unroll
    for (int i = 0; i < NDET; ++i) er[i] = ei[i] = 0.0f;
  }
  const bool has_bin = lane < 31 && base + lane < H.n_bins;
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
    const float nr = __shfl_down_sync(0xffffffffu, er[i], 1);
    const float ni = __shfl_down_sync(0xffffffffu, ei[i], 1);
    if (has_bin) {
      const float r0r = 0.5f * (er[i] + nr), r0i = 0.5f * (ei[i] + ni);
      const float r1r = (nr - er[i]) * t.iw, r1i = (ni - ei[i]) * t.iw;
      const float4 a = t.a[i];
      const float2 bb = t.bb[i];
      zr[i] += a.x * r0r - a.y * r0i + a.z * r1r - a.w * r1i;
      zi[i] += a.x * r0i + a.y * r0r + a.z * r1i + a.w * r1r;
      hh[i] += bb.x * (r0r * r0r + r0i * r0i) + 2.0f * bb.y * (r0r * r1r + r0i * r1i);
    }
  }
}

// Asynchronous global -> shared copies (cp.async, sm_80 and later): the
// lane's own table entries of a chunk, waited for one chunk later.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Layout of one stage (kernels.h het_stage_bytes): a[NDET][32] (float4),
// bb[NDET][32] (float2), iw[32], d[32].
template <int NDET>
struct HetStage {
  float4 a[NDET][32];
  float2 bb[NDET][32];
  float iw[32];
  float d[32];
};

// Lane l copies the entries of its bin 31 q + l and edge 31 q + l (the
// entries it reads itself, so no cross-lane ordering is needed).
template <int NDET>
__device__ __forceinline__ void het_stage_chunk(const HetTables& H, int q, int lane, HetStage<NDET>* st) {
  const int b = 31 * q + lane;
  if (lane < 31 && b < H.n_bins) {
#pragma unroll
    for (int i = 0; i < NDET; ++i) {
      cp_async<16>(&st->a[i][lane], H.coef + (size_t)i * H.n_bins + b);
      cp_async<8>(&st->bb[i][lane], H.coefB + (size_t)i * H.n_bins + b);
    }
    cp_async<4>(&st->iw[lane], H.inv_width + b);
  }
  if (b <= H.n_bins) cp_async<4>(&st->d[lane], H.dfe + (size_t)q * kHetChunkEdges + lane);
}

template <int NDET>
__device__ __forceinline__ void het_read_stage(const HetTables& H, int q, int lane, const HetStage<NDET>* st,
                                               HetBinData<NDET>& t) {
  const int b = 31 * q + lane;
  const bool has_bin = lane < 31 && b < H.n_bins;
  t.d = b <= H.n_bins ? st->d[lane] : 0.0f;
  t.iw = has_bin ? st->iw[lane] : 0.0f;
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
    t.a[i] = has_bin ? st->a[i][lane] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    t.bb[i] = has_bin ? st->bb[i][lane] : make_float2(0.0f, 0.0f);
  }
}

// The chunks q = first, first + stride, ... of one evaluation by one warp:
// anchored chunks (het_chunk_anc) read their table data from the warp's two
// shared-memory stages (`stage`, 2 x het_stage_bytes), filled by cp.async one
// chunk ahead, or straight from global memory when there is no room for the
// stages (stage == nullptr); exact chunks go edge by edge (het_chunk).
template <int NDET, bool TM = false>
__device__ inline void het_chunks_warp(const HetTables& H, const HetPrep<NDET>& p, const float* s_anc, int first,
                                       int stride, int lane, unsigned char* stage, float* zr, float* zi, float* hh,
                                       float2* y = nullptr) {
  const int nc = H.n_chunks;
  if (stage == nullptr) {
    for (int q = first; q < nc; q += stride) {
      const float* an = s_anc + q * kHetAncStride;
      if (an[kHetAncExact] != 0.0f) {
        het_chunk<NDET, TM>(H, p, 31 * q, lane, zr, zi, hh, y);
        continue;
      }
      const int b = 31 * q + lane;
      const bool has_bin = lane < 31 && b < H.n_bins;
      HetBinData<NDET> t;
      t.d = b <= H.n_bins ? __ldg(H.dfe + (size_t)q * kHetChunkEdges + lane) : 0.0f;
      t.iw = has_bin ? __ldg(H.inv_width + b) : 0.0f;
#pragma unroll
      for (int i = 0; i < NDET; ++i) {
        t.a[i] = has_bin ? __ldg(H.coef + (size_t)i * H.n_bins + b) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        t.bb[i] = has_bin ? __ldg(H.coefB + (size_t)i * H.n_bins + b) : make_float2(0.0f, 0.0f);
      }
      het_chunk_anc<NDET, TM>(H, p, an, q, lane, t, zr, zi, hh, y);
    }
    return;
  }
  HetStage<NDET>* st = reinterpret_cast<HetStage<NDET>*>(stage);
  if (first < nc) het_stage_chunk<NDET>(H, first, lane, st);
  cp_async_commit();
  int buf = 0;
  for (int q = first; q < nc; q += stride, buf ^= 1) {
    if (q + stride < nc) het_stage_chunk<NDET>(H, q + stride, lane, st + (buf ^ 1));
    cp_async_commit();
    cp_async_wait<1>();  // this lane's copies of chunk q have landed
    const float* an = s_anc + q * kHetAncStride;
    if (an[kHetAncExact] != 0.0f) {
      het_chunk<NDET, TM>(H, p, 31 * q, lane, zr, zi, hh, y);
    } else {
      HetBinData<NDET> t;
      het_read_stage<NDET>(H, q, lane, st + buf, t);
      het_chunk_anc<NDET, TM>(H, p, an, q, lane, t, zr, zi, hh, y);
    }
  }
  cp_async_wait<0>();
}

// Warp-sum of the lane sums (all lanes receive them).
template <int NDET>
__device__ inline void het_warp_reduce(float* zr, float* zi, float* hh) {
#pragma unroll
  for (int i = 0; i < NDET; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      zr[i] += __shfl_xor_sync(0xffffffffu, zr[i], o);
      zi[i] += __shfl_xor_sync(0xffffffffu, zi[i], o);
      hh[i] += __shfl_xor_sync(0xffffffffu, hh[i], o);
    }
}

// FP64 epilogue: plain Re Z or phase-marginalised log I0(|Z|), minus
// <h|h>/2 and <d|d>/2.
__device__ inline double het_epilogue(const LikeConst& L, double Z_re, double Z_im, double HH) {
  const double base_ll = -0.5 * HH - 0.5 * L.DD;
  if (L.phase_marg) {
    const double x = sqrt(Z_re * Z_re + Z_im * Z_im);
    return (L.fast_epilogue ? x + (double)log_i0e_f32((float)x) : log_bessel_i0(x)) + base_ll;
  }
  return Z_re + base_ll;
}

__host__ __device__ inline int het_chunks(int n_bins) { return (n_bins + 30) / 31; }

// ---------------------------------------------------------------------------
// Time pass of the time-marginalised likelihood.
// ---------------------------------------------------------------------------
constexpr int kTmNodes = 32;  // grid nodes per warp pass (lane l ends with node j0 + l)

// Log weight of one node: log I0(|Z|) with phi_c marginalised, Re Z otherwise.
__device__ __forceinline__ float tm_node_logw(const LikeConst& L, float zr, float zi) {
  if (L.phase_marg) {
    const float x = sqrtf(zr * zr + zi * zi);
    return x + log_i0e_f32(x);
  }
  return zr;
}

// One level of the halving reduction: lanes with bit O set keep the upper O
// nodes, the others the lower O, each adding its partner's copy of them.
template <int O>
__device__ __forceinline__ void tm_halve(float* ar, float* ai, int lane) {
  const bool up = (lane & O) != 0;
#pragma unroll
  for (int k = 0; k < O; ++k) {
    const float sr = up ? ar[k] : ar[k + O], si = up ? ai[k] : ai[k + O];
    const float kr = up ? ar[k + O] : ar[k], ki = up ? ai[k + O] : ai[k];
    ar[k] = kr + __shfl_xor_sync(0xffffffffu, sr, O);
    ai[k] = ki + __shfl_xor_sync(0xffffffffu, si, O);
  }
}

// One edge's inputs to the time pass: its product y_e, rotation w_e and
// frequency (double-float); an edge past the end reads as y = 0, w = 1.
struct TmEdge {
  float2 y, w;
  dfl f;
};

__device__ __forceinline__ TmEdge tm_load_edge(const HetTables& H, const float2* __restrict__ y, int e, int ne) {
  TmEdge d;
  if (e < ne) {
    d.y = y[e];
    d.w = H.tm_w[e];
    d.f = {H.edge_f[e], H.edge_f[ne + e]};
  } else {
    d.y = make_float2(0.0f, 0.0f);
    d.w = make_float2(1.0f, 0.0f);
    d.f = {0.0f, 0.0f};
  }
  return d;
}

// y_e exp(-2 pi i f_e dt): the term at the chunk's first node.
__device__ __forceinline__ float2 tm_start(const TmEdge& d, dfl dt) {
  const float twopi = 6.283185307179586f;
  float s, co;
  __sincosf(twopi * df_frac(df_mul(d.f, dt)), &s, &co);  // exp(-2 pi i f_e dt) = co - i s
  return make_float2(d.y.x * co + d.y.y * s, d.y.y * co - d.y.x * s);
}

// One warp, nodes [j0, j0 + 32): Z(dt_j) = sum_e y_e exp(-2 pi i f_e dt_j).
// Lane l takes edges l, l + 32, ... two at a time (e and e + 32, added in
// that order, so the sums are those of one edge at a time): one phasor at
// dt_j0 from the double-float phase f_e dt_j0, then a rotation by w_e per
// node (31 steps, FP32 drift ~2e-6 rad).  The next pair's loads are issued
// before the current pair's steps.  The 32 node sums are reduced across the
// warp by halving, after which lane l holds node j0 + l; returns its log
// weight (-inf past the last node).  All 32 lanes call it together.
__device__ inline float tm_nodes_warp(const LikeConst& L, const HetTables& H, const float2* __restrict__ y, int j0,
                                      int lane) {
  float ar[kTmNodes], ai[kTmNodes];
#pragma unroll
  for (int k = 0; k < kTmNodes; ++k) ar[k] = ai[k] = 0.0f;
  const dfl d0 = df_from_double(L.tm_t0 + (double)j0 * L.tm_dt);
  const int ne = H.n_bins + 1;
  TmEdge a = tm_load_edge(H, y, lane, ne), b = tm_load_edge(H, y, lane + 32, ne);
  for (int e = lane; e < ne; e += 64) {
    const TmEdge ca = a, cb = b;
    a = tm_load_edge(H, y, e + 64, ne);
    b = tm_load_edge(H, y, e + 96, ne);
    float2 u = tm_start(ca, d0), v = tm_start(cb, d0);
#pragma unroll
    for (int k = 0; k < kTmNodes; ++k) {
      ar[k] += u.x;
      ai[k] += u.y;
      ar[k] += v.x;
      ai[k] += v.y;
      const float tu = u.x * ca.w.x - u.y * ca.w.y;
      u.y = u.x * ca.w.y + u.y * ca.w.x;
      u.x = tu;
      const float tv = v.x * cb.w.x - v.y * cb.w.y;
      v.y = v.x * cb.w.y + v.y * cb.w.x;
      v.x = tv;
    }
  }
  tm_halve<16>(ar, ai, lane);
  tm_halve<8>(ar, ai, lane);
  tm_halve<4>(ar, ai, lane);
  tm_halve<2>(ar, ai, lane);
  tm_halve<1>(ar, ai, lane);
  return (j0 + lane < L.tm_n) ? tm_node_logw(L, ar[0], ai[0]) : -INFINITY;
}

// The warps of a CTA share the grid's 32-node chunks (chunk q to warp
// q mod n_warps).  Each lane keeps a running max and scaled sum of its
// nodes' exp(log weight); returns the warp's (max, sum), the same on every
// lane.  ell (optional) receives every node's log weight.
__device__ inline void tm_pass(const LikeConst& L, const HetTables& H, const float2* __restrict__ y, int warp,
                               int n_warps, int lane, float* ell, float& wm, float& ws) {
  float m = -INFINITY, s = 0.0f;
  const int nq = (L.tm_n + kTmNodes - 1) / kTmNodes;
  for (int q = warp; q < nq; q += n_warps) {
    const int j = q * kTmNodes + lane;
    const float l = tm_nodes_warp(L, H, y, q * kTmNodes, lane);
    if (j < L.tm_n) {
      if (ell) ell[j] = l;
      if (l > m) {
        s = s * __expf(m - l) + 1.0f;
        m = l;
      } else {
        s += __expf(l - m);
      }
    }
  }
  float M = m;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));
  float S = (m > -INFINITY) ? s * __expf(m - M) : 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
  wm = M;
  ws = S;
}

// The gather's per-piece partial sums follow the grid and its twiddles.
__device__ __forceinline__ float2* tm_nufft_parts(const LikeConst& L, float2* g) { return g + 2 * L.tm_M; }

// Gather of the non-uniform FFT's grid values b_l = sum_e w_le c_e (the
// whole block).  A grid point's entries are consecutive edges, cut into
// pieces of at most kNufftPiece entries; lane t sums pieces t, t + nt, ...
// (all of a piece's weight loads issued together) into part[], then thread
// t combines the pieces of grid points t, t + nt, ... in order.  Fixed sum
// orders: deterministic.  Grid points without entries are zeroed.
__device__ inline void nufft_gather(const LikeConst& L, const HetTables& H, const float2* y, float2* g,
                                    float2* part, int lg) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int l = tid; l < L.tm_M; l += nt) g[l] = make_float2(0.0f, 0.0f);
  // the descriptors of this thread's first four pieces, loaded together
  constexpr int kPre = 4;
  int4 dp[kPre];
#pragma unroll
  for (int r = 0; r < kPre; ++r)
    dp[r] = tid + r * nt < L.tm_pieces ? __ldg(&H.nu_piece[tid + r * nt]) : make_int4(0, 0, 0, 0);
  for (int p = tid, r = 0; p < L.tm_pieces; p += nt, ++r) {
    int4 d = dp[0];
#pragma unroll
    for (int u = 1; u < kPre; ++u)
      if (r == u) d = dp[u];
    if (r >= kPre) d = __ldg(&H.nu_piece[p]);
    float w[kNufftPiece];
#pragma unroll
    for (int i = 0; i < kNufftPiece; ++i) w[i] = i < d.y ? __ldg(&H.nu_wt[d.x + i]) : 0.0f;
    float br = 0.0f, bi = 0.0f;
#pragma unroll
    for (int i = 0; i < kNufftPiece; ++i)
      if (i < d.y) {
        const float2 c = y[d.z + i];
        br = fmaf(w[i], c.x, br);
        bi = fmaf(w[i], c.y, bi);
      }
    part[p] = make_float2(br, bi);
  }
  __syncthreads();
  for (int q = tid; q < L.tm_points; q += nt) {
    const int4 d = __ldg(&H.nu_point[q]);
    float br = 0.0f, bi = 0.0f;
    for (int i = 0; i < d.z; ++i) {
      const float2 v = part[d.y + i];
      br += v.x;
      bi += v.y;
    }
    g[__brev((unsigned)d.x) >> (32 - lg)] = make_float2(br, bi);
  }
}

// The same time pass by non-uniform FFT (tables of het_nufft_tables): the
// edge products become c_e = y_e exp(-2 pi i f_e dt_ref) (double-float phase;
// y is overwritten), every grid point gathers its kernel-weighted c_e in a
// fixed order into bit-reversed position, a radix-2 FFT with exponent
// +2 pi i runs in shared memory, and node j takes Z_j = X[(j - j0) mod M] /
// Phi(j - j0).  Nodes are assigned to warps and lanes as in tm_pass, so the
// (max, sum) pairs and ell have the same layout.  Every thread of the CTA
// calls it (it synchronises the CTA).  Cost per evaluation ~W (N_b + 1)
// multiply-adds for the gather and (M/2) log2 M butterflies, against
// (N_b + 1) N_t terms for the direct sum.
__device__ inline void tm_pass_nufft(const LikeConst& L, const HetTables& H, const float2* y, float2* g,
                                     const float2* tw, int warp, int n_warps, int lane, float* ell, float& wm,
                                     float& ws) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int M = L.tm_M;
  // y holds c_e (the edge weights carry the reference rotation)
  const int lg = __ffs(M) - 1;
  nufft_gather(L, H, y, g, tm_nufft_parts(L, g), lg);
  __syncthreads();
  // radix-2 stages of spans 1..16 inside 32-point blocks in registers (warp
  // shuffles: no shared-memory bank conflicts, no block barriers), then the
  // wider spans through shared memory
  for (int blk = warp; blk < M / 32; blk += n_warps) {
    const int at = blk * 32 + lane;
    float2 x = g[at];
#pragma unroll
    for (int half = 1; half < 32; half <<= 1) {
      const float2 w = tw[half - 1 + (lane & (half - 1))];
      const float pr = __shfl_xor_sync(0xffffffffu, x.x, half), pi = __shfl_xor_sync(0xffffffffu, x.y, half);
      if ((lane & half) == 0)  // lower point: x + w partner
        x = make_float2(x.x + (w.x * pr - w.y * pi), x.y + (w.x * pi + w.y * pr));
      else  // upper point: partner - w x
        x = make_float2(pr - (w.x * x.x - w.y * x.y), pi - (w.x * x.y + w.y * x.x));
    }
    g[at] = x;
  }
  __syncthreads();
  for (int half = 32; half < M; half <<= 1) {
    for (int b = tid; b < M / 2; b += nt) {
      const int pos = b & (half - 1), i = ((b - pos) << 1) + pos, j = i + half;
      const float2 w = tw[half - 1 + pos];
      const float2 xj = g[j], xi = g[i];
      const float tr = w.x * xj.x - w.y * xj.y, ti = w.x * xj.y + w.y * xj.x;
      g[j] = make_float2(xi.x - tr, xi.y - ti);
      g[i] = make_float2(xi.x + tr, xi.y + ti);
    }
    __syncthreads();
  }
  float m = -INFINITY, s = 0.0f;
  const int nq = (L.tm_n + kTmNodes - 1) / kTmNodes;
  for (int q = warp; q < nq; q += n_warps) {
    const int j = q * kTmNodes + lane;
    if (j < L.tm_n) {
      const int mi = j - L.tm_j0;
      const float2 z = g[mi < 0 ? mi + M : mi];
      const float cr = H.nu_corr[j];
      const float l = tm_node_logw(L, z.x * cr, z.y * cr);
      if (ell) ell[j] = l;
      if (l > m) {
        s = s * __expf(m - l) + 1.0f;
        m = l;
      } else {
        s += __expf(l - m);
      }
    }
  }
  float Mx = m;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) Mx = fmaxf(Mx, __shfl_xor_sync(0xffffffffu, Mx, o));
  float S = (m > -INFINITY) ? s * __expf(m - Mx) : 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
  wm = Mx;
  ws = S;
}

// The NUFFT grid's place in shared memory: after the N_b + 1 edge products;
// its M stage-major twiddles follow the grid (tm_nufft_tw).
__device__ __forceinline__ float2* tm_nufft_grid(unsigned char* smem, int n_bins) {
  return reinterpret_cast<float2*>(smem + ((((size_t)n_bins + 1) * 2 * sizeof(float) + 15) / 16 * 16));
}
__device__ __forceinline__ float2* tm_nufft_tw(unsigned char* smem, int n_bins, int M) {
  return tm_nufft_grid(smem, n_bins) + M;
}
// Copy of the twiddle table into shared memory (whole block).
__device__ __forceinline__ void tm_load_twiddles(const LikeConst& L, const HetTables& H, unsigned char* smem,
                                                 int n_bins) {
  float2* tw = tm_nufft_tw(smem, n_bins, L.tm_M);
  for (int k = threadIdx.x; k < L.tm_M; k += blockDim.x) tw[k] = __ldg(&H.nu_tw[k]);
}

// Time-marginalised logL from the warps' (max, sum) pairs (warp order) and
// the network <h|h>: log((1/N_t) sum_j exp(l_j)) - <h|h>/2 - <d|d>/2.
__device__ inline double tm_finish(const LikeConst& L, const float (*wms)[2], int n_warps, double HH) {
  float M = -INFINITY;
  for (int w = 0; w < n_warps; ++w) M = fmaxf(M, wms[w][0]);
  double S = 0.0;
  for (int w = 0; w < n_warps; ++w)
    if (wms[w][0] > -INFINITY) S += (double)wms[w][1] * exp((double)wms[w][0] - (double)M);
  return (double)M + log(S) - log((double)L.tm_n) - 0.5 * HH - 0.5 * L.DD;
}

// Per-detector sums cached for projection-only evaluations: (Z_i / C_i) /
// inv_scale_i as the chain's kappa, and <h|h>_i / |C_i|^2 times A1^2 (the
// heterodyned Z_i is linear and <h|h>_i quadratic in C_i).
__device__ inline void het_cache(const LikeConst& L, const EvalRecord& r, int i, double zr, double zi, double hh,
                                 double* kap2, double* vv) {
  const double cr = r.cre[i], ci = r.cim[i], c2 = cr * cr + ci * ci;
  if (c2 > 0.0) {
    const double ic2 = 1.0 / c2, k = ic2 / L.inv_scale[i];
    kap2[0] = (zr * cr + zi * ci) * k;
    kap2[1] = (zi * cr - zr * ci) * k;
    *vv = hh * ic2 * (L.amp1 * L.amp1);
  } else {
    kap2[0] = kap2[1] = 0.0;
    *vv = 0.0;
  }
}

// One warp evaluates the heterodyned logL of record r (all lanes return it);
// optionally the per-detector cache of het_cache (lane 0 writes it).
template <int NDET>
__device__ inline double het_loglike_warp(const LikeConst& L, const HetTables& H, const EvalRecord& r, int lane,
                                          double* kap_out = nullptr, double* vv_out = nullptr) {
  if (!r.valid) {
    if (lane == 0 && kap_out)
      for (int j = 0; j < 2 * SWIG_MAX_DET; ++j) kap_out[j] = 0.0;
    if (lane == 0 && vv_out)
      for (int i = 0; i < SWIG_MAX_DET; ++i) vv_out[i] = 0.0;
    return -INFINITY;
  }
  HetPrep<NDET> p;
  het_prepare<NDET>(L, H, r, p);
  float zr[NDET], zi[NDET], hh[NDET];
#pragma unroll
  for (int i = 0; i < NDET; ++i) zr[i] = zi[i] = hh[i] = 0.0f;
  const int nc = het_chunks(H.n_bins);
  for (int q = 0; q < nc; ++q) het_chunk<NDET>(H, p, 31 * q, lane, zr, zi, hh);
  het_warp_reduce<NDET>(zr, zi, hh);
  double Z_re = 0.0, Z_im = 0.0, HH = 0.0;
#pragma unroll
  for (int i = 0; i < NDET; ++i) {
    Z_re += (double)zr[i];
    Z_im += (double)zi[i];
    HH += (double)hh[i];
  }
  if (lane == 0 && kap_out && vv_out) {
    for (int i = 0; i < SWIG_MAX_DET; ++i) {
      kap_out[2 * i] = kap_out[2 * i + 1] = 0.0;
      vv_out[i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < NDET; ++i) het_cache(L, r, i, zr[i], zi[i], hh[i], kap_out + 2 * i, vv_out + i);
  }
  return het_epilogue(L, Z_re, Z_im, HH);
}

}  // namespace swig
