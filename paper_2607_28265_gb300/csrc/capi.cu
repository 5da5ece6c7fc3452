// C-ABI of libswig: context management, problem definition, host-side FP64
// preparation (data weighting, tile planning) and the likelihood entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <iterator>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"
#include "device_common.cuh"
#include "kernels.h"
#include "swig.h"

using namespace swig;

namespace {

thread_local std::string g_create_error;

int fail(swig_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CUDA_TRY(ctx, call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? SWIG_E_NOMEM : SWIG_E_CUDA,  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    }                                                                                   \
  } while (0)

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// Compensated (Neumaier) summation for host reductions over the grid.
struct NSum {
  double s = 0.0, c = 0.0;
  void add(double x) {
    const double t = s + x;
    if (std::fabs(s) >= std::fabs(x))
      c += (s - t) + x;
    else
      c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

// n-th derivative of f^p (ln f)^lg at f as coefficients: f^(p-n) (a ln f + b).
double basis_derivative(double p, int lg, int n, double f) {
  if (!lg) {
    double fall = 1.0;
    for (int i = 0; i < n; ++i) fall *= (p - i);
    return fall * std::pow(f, p - n);
  }
  double a = 1.0, b = 0.0;
  for (int i = 0; i < n; ++i) {
    const double na = (p - i) * a, nb = (p - i) * b + a;
    a = na;
    b = nb;
  }
  return std::pow(f, p - n) * (a * std::log(f) + b);
}

// |n-th derivative| bound on [f0, f1] (monotone power times log factor).
double basis_derivative_bound(double p, int lg, int n, double f0, double f1) {
  if (!lg) {
    double fall = 1.0;
    for (int i = 0; i < n; ++i) fall *= (p - i);
    return std::fabs(fall) * std::max(std::pow(f0, p - n), std::pow(f1, p - n));
  }
  double a = 1.0, b = 0.0;
  for (int i = 0; i < n; ++i) {
    const double na = (p - i) * a, nb = (p - i) * b + a;
    a = na;
    b = nb;
  }
  const double lmax = std::max(std::fabs(std::log(f0)), std::fabs(std::log(f1)));
  return std::max(std::pow(f0, p - n), std::pow(f1, p - n)) * (std::fabs(a) * lmax + std::fabs(b));
}

const double kBasisPow[NBASIS] = {-5.0 / 3.0, -1.0, -2.0 / 3.0, -1.0 / 3.0, 0.0, 1.0 / 3.0,
                                  1.0 / 3.0,  2.0 / 3.0, 5.0 / 3.0, 7.0 / 3.0, 0.0};
const int kBasisLog[NBASIS] = {0, 0, 0, 0, 1, 0, 1, 0, 0, 0, 0};

void split_df(double x, float* hi, float* lo) {
  const float h = (float)x;
  *hi = h;
  *lo = (float)(x - (double)h);
}

// Largest |c_j| over the corners of the intrinsic prior box (x1.25 margin).
void coefficient_bounds(const swig_ctx* c, double* cmax) {
  double lo[6], hi[6];
  const double dlo[6] = {0.87, 0.125, -0.1, -0.1, 0.0, 0.0}, dhi[6] = {3.0, 1.0, 0.1, 0.1, 5000.0, 5000.0};
  for (int i = 0; i < 6; ++i) {
    lo[i] = dlo[i];
    hi[i] = dhi[i];
    if (c->prior_set) {
      const swig_param& p = c->params[i];
      if (p.mode == SWIG_MODE_FIXED) {
        lo[i] = hi[i] = p.value;
      } else if (p.mode == SWIG_MODE_SAMPLE) {
        lo[i] = p.lo;
        hi[i] = p.hi;
      }
    }
  }
  for (int j = 0; j < NBASIS; ++j) cmax[j] = 0.0;
  for (int m = 0; m < 64; ++m) {
    double v[6];
    for (int i = 0; i < 6; ++i) v[i] = (m >> i & 1) ? hi[i] : lo[i];
    double cc[NBASIS];
    taylorf2_basis_coeffs(v[0], v[1], v[2], v[3], v[4], v[5], cc);
    for (int j = 0; j < NBASIS; ++j) cmax[j] = std::max(cmax[j], std::fabs(cc[j]));
  }
  for (int j = 0; j < NBASIS; ++j) cmax[j] *= 1.25;
}

// Tiles of 2^m bins (1 .. kMaxTileBins) whose degree-kTaylorDeg Taylor
// remainder of the phase (in cycles) stays below `eps` over the prior box.
// Tiles up to 32 bins start at a multiple of their size (so they never cross a
// 32-bin chunk); larger tiles start on a chunk boundary.
void plan_tiles(const swig_ctx* c, std::vector<TileInfo>& tiles, std::vector<TileBasis>& basis) {
  double cmax[NBASIS];
  coefficient_bounds(c, cmax);
  const double eps = 1e-8;
  const int n = (int)c->n_bins;
  const int order = kTaylorDeg + 1;
  double fact = 1.0;
  for (int i = 2; i <= order; ++i) fact *= i;
  tiles.clear();
  basis.clear();
  int k = 0;
  while (k < n) {
    int T = 1;
    while (T * 2 <= kMaxTileBins) {
      const int T2 = T * 2;
      if (T2 <= kChunk && k % T2 != 0) break;
      if (T2 > kChunk && k % kChunk != 0) break;
      const double fa = (double)(c->k_min + k) * c->df, fb = fa + T2 * c->df;
      double R = 0.0;
      for (int j = 0; j < NBASIS - 1; ++j)
        R += cmax[j] * basis_derivative_bound(kBasisPow[j], kBasisLog[j], order, fa, fb);
      R *= std::pow(T2 * c->df, order) / fact;
      if (R > eps) break;
      T = T2;
    }
    TileInfo ti;
    ti.k0 = k;
    ti.nbins = std::min(T, n - k);
    const double fa = (double)(c->k_min + k) * c->df;
    split_df(fa, &ti.fa_hi, &ti.fa_lo);
    int span = 1, bits = 0;
    while (span < ti.nbins) {
      span *= 2;
      ++bits;
    }
    ti.inv_T = 1.0f / (float)span;
    ti.split_bits = bits;
    TileBasis tb;
    for (int j = 0; j < NBASIS; ++j) {
      double val, slope;
      double poly[kNumPoly];
      if (j == B_ONE) {
        val = 1.0;
        slope = 0.0;
        for (int m = 0; m < kNumPoly; ++m) poly[m] = 0.0;
      } else {
        val = basis_derivative(kBasisPow[j], kBasisLog[j], 0, fa);
        slope = basis_derivative(kBasisPow[j], kBasisLog[j], 1, fa) * c->df;
        double nf = 1.0;
        for (int m = 0; m < kNumPoly; ++m) {
          const int nn = m + 2;
          nf *= nn;
          poly[m] = basis_derivative(kBasisPow[j], kBasisLog[j], nn, fa) * std::pow(c->df * span, nn) / nf;
        }
      }
      split_df(val, &tb.val_hi[j], &tb.val_lo[j]);
      split_df(slope, &tb.slope_hi[j], &tb.slope_lo[j]);
      for (int m = 0; m < kNumPoly; ++m) tb.poly[m][j] = (float)poly[m];
    }
    tiles.push_back(ti);
    basis.push_back(tb);
    k += ti.nbins;
  }
}

void free_scratch(DeviceBuffers& B) {
  dfree(B.rec);
  dfree(B.anchors);
  dfree(B.partials32);
  dfree(B.partials64);
  dfree(B.theta);
  dfree(B.out);
  dfree(B.u);
  B.cap = 0;
}

void free_problem(DeviceBuffers& B) {
  dfree(B.data32);
  dfree(B.data64);
  dfree(B.ftab);
  dfree(B.tiles);
  dfree(B.basis);
  dfree(B.slice_begin);
  dfree(B.bin_tile);
  dfree(B.prior);
  dfree(B.piece_begin);
  dfree(B.slice_piece);
  dfree(B.het_edge_basis);
  dfree(B.het_edge_f);
  dfree(B.het_inv_width);
  dfree(B.het_chunk);
  dfree(B.het_dfe);
  B.het_nc = 0;
  dfree(B.het_coef);
  dfree(B.het_coefB);
  dfree(B.het_fid);
  dfree(B.het_tm_g);
  dfree(B.het_tm_w);
  dfree(B.het_nu_wt);
  dfree(B.het_nu_corr);
  dfree(B.het_nu_tw);
  dfree(B.het_nu_piece);
  dfree(B.het_nu_point);
  B.het_nb = 0;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on the
// three-term recurrence of the Legendre polynomials, Golub-Welsch-free).
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double dz = p1 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

// Bin edges (grid indices) of the heterodyned likelihood.  spacing 0: equal
// increments of the maximum dephasing g(f) = sum_gamma sign(gamma) (f/f*)^gamma,
// gamma in {-5/3, -2/3, 1, 5/3, 7/3}, f* = f_lo for gamma < 0 and f_hi
// otherwise (Zackay, Dai & Venumadhav 2018); spacing 1: geometric.  Targets are
// snapped to the first grid frequency at or above them; duplicates dropped.
std::vector<int> het_edge_indices(const std::vector<double>& f, int nb, int spacing) {
  const int n = (int)f.size();
  std::vector<double> g(n);
  const double f_lo = f.front(), f_hi = f.back();
  if (spacing == 0) {
    const double gam[5] = {-5.0 / 3.0, -2.0 / 3.0, 1.0, 5.0 / 3.0, 7.0 / 3.0};
    for (int k = 0; k < n; ++k) {
      double v = 0.0;
      for (double gm : gam) {
        const double fs = gm < 0 ? f_lo : f_hi;
        v += (gm < 0 ? -1.0 : 1.0) * std::pow(f[k] / fs, gm);
      }
      g[k] = v;
    }
  } else {
    g = f;
  }
  std::vector<int> idx;
  const double ga = g.front(), gb = g.back();
  for (int i = 0; i <= nb; ++i) {
    double t;
    if (spacing == 0) {
      t = (i == nb) ? gb : ga + i * ((gb - ga) / nb);
    } else {
      const double l0 = std::log10(f_lo), l1 = std::log10(f_hi);
      t = (i == 0) ? f_lo : (i == nb) ? f_hi : std::pow(10.0, l0 + i * ((l1 - l0) / nb));
    }
    int k = (int)(std::lower_bound(g.begin(), g.end(), t) - g.begin());
    if (i == 0) k = 0;
    if (i == nb) k = n - 1;
    k = std::min(k, n - 1);
    if (idx.empty() || k > idx.back()) idx.push_back(k);
  }
  if (idx.back() != n - 1) idx.push_back(n - 1);
  return idx;
}

// Weighted data of the full-grid likelihood (Eq. 2 expanded): D_i(k) =
// 4 df conj(d_i) f^-7/6 / S_i (dre, dim: [n_det][n_bins]), K_i = 4 df sum
// f^-7/3 / S_i, <d|d> summed over the detectors (compensated FP64 sums), and
// the largest |D_i| of each detector (the mixed path's data scale).
void weight_data(const swig_ctx* c, int n_det, std::vector<double>& dre, std::vector<double>& dim, double* K,
                 double* dd, double* dmax) {
  const int64_t n = c->n_bins;
  dre.assign((size_t)n_det * n, 0.0);
  dim.assign((size_t)n_det * n, 0.0);
  NSum dsum;
  for (int i = 0; i < n_det; ++i) {
    NSum Ks;
    dmax[i] = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      const double f = (double)(c->k_min + k) * c->df;
      const double w = 4.0 * c->df / c->psd[i][k];
      const double re = c->data[i][2 * k], im = c->data[i][2 * k + 1];
      const double a = w * std::pow(f, -7.0 / 6.0);
      dre[i * n + k] = a * re;
      dim[i * n + k] = -a * im;
      Ks.add(w * std::pow(f, -7.0 / 3.0));
      dsum.add(w * (re * re + im * im));
      dmax[i] = std::max(dmax[i], std::hypot(re, im) * a);
    }
    K[i] = Ks.value();
  }
  *dd = dsum.value();
}

// Summary data of the heterodyned likelihood (Sec. 3.4) per detector and bin:
// bin b holds the grid bins idx[b] <= k < idx[b + 1] (the last bin also the
// last grid bin); with the centre f_c and w = 4 df / S,
//   A0 = sum conj(d) h0 w,  A1 = sum conj(d) h0 w (f - f_c),
//   B0 = sum |h0|^2 w,      B1 = sum |h0|^2 w (f - f_c),
// compensated FP64 sums stored FP32 (coef: A0, A1; coefB: B0, B1) and kept in
// FP64 in a01 (A0.re, A0.im, A1.re, A1.im).  data[i] holds re, im interleaved;
// h0 is [n_det][n] on the grid.
void het_summary(const std::vector<double>& f, const std::vector<int>& idx, int nb, int n_det, double df,
                 const std::vector<double>* data, const std::vector<double>* psd, const std::vector<double2>& h0,
                 std::vector<float4>& coef, std::vector<float2>& coefB, std::vector<double>& a01) {
  const int n = (int)f.size();
  coef.assign((size_t)n_det * nb, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
  coefB.assign((size_t)n_det * nb, make_float2(0.0f, 0.0f));
  a01.assign((size_t)n_det * nb * 4, 0.0);
  for (int i = 0; i < n_det; ++i) {
    for (int b = 0; b < nb; ++b) {
      const int k_end = (b == nb - 1) ? n : idx[b + 1];
      const double fc = 0.5 * (f[idx[b]] + f[idx[b + 1]]);
      NSum a0r, a0i, a1r, a1i, b0, b1;
      for (int k = idx[b]; k < k_end; ++k) {
        const double w = 4.0 * df / psd[i][k];
        const double dr = data[i][2 * k], di = data[i][2 * k + 1];
        const double hr = h0[(size_t)i * n + k].x, hi = h0[(size_t)i * n + k].y;
        const double pr = (dr * hr + di * hi) * w, pi = (dr * hi - di * hr) * w;  // conj(d) h0 w
        const double hh = (hr * hr + hi * hi) * w, off = f[k] - fc;
        a0r.add(pr);
        a0i.add(pi);
        a1r.add(pr * off);
        a1i.add(pi * off);
        b0.add(hh);
        b1.add(hh * off);
      }
      coef[(size_t)i * nb + b] = make_float4((float)a0r.value(), (float)a0i.value(), (float)a1r.value(), (float)a1i.value());
      double* a = &a01[((size_t)i * nb + b) * 4];
      a[0] = a0r.value();
      a[1] = a0i.value();
      a[2] = a1r.value();
      a[3] = a1i.value();
      coefB[(size_t)i * nb + b] = make_float2((float)b0.value(), (float)b1.value());
    }
  }
}

// Tables of the time-marginalised heterodyne, in FP64 and stored FP32: the
// edge weights g_ie (Z_i = sum_e g_ie r_i(e): the bin above an edge gives
// A0/2 - A1/w, the bin below A0/2 + A1/w) from a01 = (A0.re, A0.im, A1.re,
// A1.im) per detector and bin, and the rotation exp(-2 pi i f_e dt) of each
// edge per grid step.  f[idx[q]] is the frequency of edge q.
void het_tm_tables(const std::vector<double>& a01, const std::vector<double>& f, const std::vector<int>& idx,
                   int nb, int n_det, double dt, std::vector<float2>& g, std::vector<float2>& w, double dref = 0.0) {
  const size_t ne = (size_t)nb + 1;
  g.assign((size_t)n_det * ne, make_float2(0.0f, 0.0f));
  w.assign(ne, make_float2(0.0f, 0.0f));
  for (int i = 0; i < n_det; ++i)
    for (int q = 0; q <= nb; ++q) {
      double gr = 0.0, gi = 0.0;
      if (q < nb) {
        const double* a = &a01[((size_t)i * nb + q) * 4];
        const double iw = 1.0 / (f[idx[q + 1]] - f[idx[q]]);
        gr += 0.5 * a[0] - a[2] * iw;
        gi += 0.5 * a[1] - a[3] * iw;
      }
      if (q > 0) {
        const double* a = &a01[((size_t)i * nb + q - 1) * 4];
        const double iw = 1.0 / (f[idx[q]] - f[idx[q - 1]]);
        gr += 0.5 * a[0] + a[2] * iw;
        gi += 0.5 * a[1] + a[3] * iw;
      }
      if (dref != 0.0) {  // times exp(-2 pi i f_e dref), the non-uniform FFT's reference rotation
        double ph = f[idx[q]] * dref;
        ph -= std::nearbyint(ph);
        const double cr = std::cos(2.0 * kPi * ph), ci = -std::sin(2.0 * kPi * ph);
        const double tr = gr * cr - gi * ci;
        gi = gr * ci + gi * cr;
        gr = tr;
      }
      g[(size_t)i * ne + q] = make_float2((float)gr, (float)gi);
    }
  for (int q = 0; q <= nb; ++q) {
    double ph = f[idx[q]] * dt;
    ph -= std::nearbyint(ph);
    w[q] = make_float2((float)std::cos(2.0 * kPi * ph), (float)-std::sin(2.0 * kPi * ph));
  }
}

// Tables of the time pass by non-uniform FFT (type 1; Dutt & Rokhlin 1993,
// Greengard & Lee 2004) with the "exponential of semicircle" kernel of
// Barnett, Magland & af Klinteberg (2019): with u_e = f_e dt (cycles per
// node) and the reference shift dt_ref = t_0 + j0 dt of node j0,
//   Z(dt_ref + m dt) = sum_e c_e exp(2 pi i xi_e m),  xi_e = frac(-u_e),
//   c_e = y_e exp(-2 pi i f_e dt_ref),
// for m = j - j0.  The c_e are spread onto M >= 2 N_t grid points with
// phi(z) = exp(beta (sqrt(1 - (2 z / W)^2) - 1)), |z| <= W / 2 (z in grid
// units, W points, beta = 2.3 W), b_l = sum_e c_e phi(l - M xi_e) (periodic);
// then Z_m = [sum_l b_l exp(2 pi i m l / M)] / Phi(m), Phi(m) the kernel's
// Fourier integral.  The spreading is stored as a gather list per grid point
// (edges in increasing order) so that every sum has a fixed order.
// Outputs: M, j0, ptr [M + 1] (entries of each grid point), edge [M] (its
// first edge; its edges are consecutive), weight per entry, corr [N_t] = 1 /
// Phi(j - j0), twiddles [M / 2] = exp(2 pi i k / M); ptr comes back empty
// (and the direct sum is used) if some grid point's edges are not consecutive.
void het_nufft_tables(const std::vector<double>& fe, int n_t, double dt, int width, int* M_out, int* j0_out,
                      std::vector<int>& ptr, std::vector<int>& edge, std::vector<float>& wt,
                      std::vector<float>& corr, std::vector<float2>& tw) {
  int M = 1;
  while (M < 2 * n_t) M <<= 1;
  const int j0 = n_t / 2;
  const double W = (double)width, beta = 2.3 * W;
  auto phi = [&](double z) {
    const double t = 2.0 * z / W;
    return std::fabs(t) > 1.0 ? 0.0 : std::exp(beta * (std::sqrt(1.0 - t * t) - 1.0));
  };
  const int ne = (int)fe.size();
  std::vector<std::vector<std::pair<int, float>>> lists(M);
  for (int e = 0; e < ne; ++e) {
    double u = fe[e] * dt;
    double xi = -u - std::floor(-u);  // frac(-u) in [0, 1)
    const double cpos = xi * M;
    const int l_lo = (int)std::ceil(cpos - 0.5 * W), l_hi = (int)std::floor(cpos + 0.5 * W);
    for (int l = l_lo; l <= l_hi; ++l) {
      const double v = phi((double)l - cpos);
      if (v == 0.0) continue;
      const int lw = ((l % M) + M) % M;
      lists[lw].push_back({e, (float)v});
    }
  }
  // edge[l] = the first edge of grid point l: its edges are consecutive (xi_e
  // is monotone in e), so the weights alone are stored per entry
  ptr.assign(M + 1, 0);
  edge.assign(M, 0);
  wt.clear();
  for (int l = 0; l < M; ++l) {
    const auto& li = lists[l];
    if (!li.empty()) {
      edge[l] = li.front().first;
      for (size_t q = 0; q < li.size(); ++q) {
        if (li[q].first != li.front().first + (int)q) {  // not consecutive: fall back to no NUFFT tables
          ptr.clear();
          return;
        }
        wt.push_back(li[q].second);
      }
    }
    ptr[l + 1] = (int)wt.size();
  }
  // Phi(m) = int phi(z) cos(2 pi m z / M) dz: twice the integral over the
  // half-support (the integrand is even), 8 panels of Gauss-Legendre
  double gx[kGaussLegendre], gw[kGaussLegendre];
  gauss_legendre(kGaussLegendre, gx, gw);
  corr.assign(n_t, 0.0f);
  for (int j = 0; j < n_t; ++j) {
    const int m = j - j0;
    double acc = 0.0;
    const int pieces = 8;  // the half-support [0, W/2] in 8 panels
    for (int pc = 0; pc < pieces; ++pc) {
      const double a = 0.5 * W * pc / pieces, b = 0.5 * W * (pc + 1) / pieces;
      for (int k = 0; k < kGaussLegendre; ++k) {
        const double z = 0.5 * (a + b) + 0.5 * (b - a) * gx[k];
        acc += 0.5 * (b - a) * gw[k] * phi(z) * std::cos(2.0 * kPi * m * z / M);
      }
    }
    corr[j] = (float)(1.0 / (2.0 * acc));
  }
  tw.resize(M / 2);
  for (int k = 0; k < M / 2; ++k)
    tw[k] = make_float2((float)std::cos(2.0 * kPi * k / M), (float)std::sin(2.0 * kPi * k / M));
  *M_out = M;
  *j0_out = j0;
}

}  // namespace

namespace swig {

// Summary data of the heterodyned likelihood (host FP64 from the device FP64
// fiducial waveform) and the per-edge basis tables.
// Twiddles of the time pass's radix-2 FFT stage by stage: span h (1, 2, 4,
// ..., M / 2) at h - 1 + p for p < h holds exp(2 pi i p / (2 h)), taken from
// the plain table tw[k] = exp(2 pi i k / M) at k = p M / (2 h), so that every
// stage reads consecutive entries.  M entries (the last unused).
std::vector<float2> nufft_stage_twiddles(const std::vector<float2>& tw, int M) {
  std::vector<float2> tws(M, make_float2(0.0f, 0.0f));
  for (int h = 1; h < M; h <<= 1)
    for (int q = 0; q < h; ++q) tws[h - 1 + q] = tw[(size_t)q * (M / (2 * h))];
  return tws;
}

// Gather pieces of the time pass's non-uniform FFT: each grid point's
// entries (ptr[l] .. ptr[l + 1], consecutive edges from edge[l]) in runs of
// at most kNufftPiece, piece = (first entry, entries, first edge, 0), and the
// grid points with entries, point = (grid point, first piece, pieces, 0).
void nufft_pieces(const std::vector<int>& ptr, const std::vector<int>& edge, int M, std::vector<int4>& piece,
                  std::vector<int4>& point) {
  piece.clear();
  point.clear();
  for (int l = 0; l < M; ++l) {
    const int n = ptr[l + 1] - ptr[l];
    if (n == 0) continue;
    point.push_back(make_int4(l, (int)piece.size(), (n + kNufftPiece - 1) / kNufftPiece, 0));
    for (int o = 0; o < n; o += kNufftPiece)
      piece.push_back(make_int4(ptr[l] + o, std::min(kNufftPiece, n - o), edge[l] + o, 0));
  }
}

// Chunk anchor tables of the heterodyned contraction (kernels.h
// HetChunkRow): chunk q holds edges 31 q .. 31 q + 31 (f[idx[e]]), anchored
// at its first edge f_a with span S = f_last - f_a; rows: basis values and
// first derivatives times S (double-float), derivatives of orders
// 2..kHetTaylorDeg times S^n / n! (float), f_a, 1 / S, and the order-11
// remainder bound per unit coefficient, max |phi_j^(11)| S^11 / 11! over the
// chunk.  dfe[32 q + l] = f_e - f_a.  Returns the number of chunks.
int het_chunk_tables(const std::vector<double>& f, const std::vector<int>& idx, int nb, std::vector<float>& ct,
                     std::vector<float>& dfe) {
  const int nc = (nb + 30) / 31;
  ct.assign((size_t)HC_ROWS * nc, 0.0f);
  dfe.assign((size_t)nc * kHetChunkEdges, 0.0f);
  {
    const int order = kHetTaylorDeg + 1;
    double fact = 1.0;
    for (int i = 2; i <= order; ++i) fact *= i;
    for (int q = 0; q < nc; ++q) {
      const int e0 = 31 * q, e1 = std::min(31 * q + 31, nb);
      const double fa = f[idx[e0]], fb = f[idx[e1]], span = fb - fa;
      auto put = [&](int row, double v) { ct[(size_t)row * nc + q] = (float)v; };
      float hi, lo;
      split_df(fa, &hi, &lo);
      put(HC_FA_HI, hi);
      put(HC_FA_LO, lo);
      put(HC_INV_S, span > 0.0 ? 1.0 / span : 0.0);
      for (int j = 0; j < NBASIS; ++j) {
        const bool one = j == B_ONE;
        // remainder bound per unit |c_j - c0_j| (the device sums it per evaluation)
        put(HC_BND + j,
            one ? 0.0 : basis_derivative_bound(kBasisPow[j], kBasisLog[j], order, fa, fb) * std::pow(span, order) / fact);
        split_df(one ? 1.0 : basis_derivative(kBasisPow[j], kBasisLog[j], 0, fa), &hi, &lo);
        put(HC_VAL_HI + j, hi);
        put(HC_VAL_LO + j, lo);
        split_df(one ? 0.0 : basis_derivative(kBasisPow[j], kBasisLog[j], 1, fa) * span, &hi, &lo);
        put(HC_D1_HI + j, hi);
        put(HC_D1_LO + j, lo);
        double nf = 1.0;
        for (int m = 0; m < kHetPoly; ++m) {
          const int nn = m + 2;
          nf *= nn;
          put(HC_POLY + m * NBASIS + j,
              one ? 0.0 : basis_derivative(kBasisPow[j], kBasisLog[j], nn, fa) * std::pow(span, nn) / nf);
        }
      }
      for (int l = 0; l < kHetChunkEdges && e0 + l <= nb; ++l) dfe[(size_t)q * kHetChunkEdges + l] = (float)(f[idx[e0 + l]] - fa);
    }
  }
  return nc;
}

int prepare_het(swig_ctx* c) {
  LikeConst& L = c->L;
  DeviceBuffers& B = c->B;
  const int n = L.n_bins, n_det = L.n_det;
  std::vector<double> f(n);
  for (int k = 0; k < n; ++k) f[k] = (double)(c->k_min + k) * c->df;
  const std::vector<int> idx = het_edge_indices(f, c->cfg.het_bins, c->cfg.het_spacing);
  const int nb = (int)idx.size() - 1;
  if (nb < 1) return fail(c, SWIG_E_ARG, "heterodyne needs at least one bin");
  double th[SWIG_N_PARAMS];
  for (int j = 0; j < SWIG_N_PARAMS; ++j) th[j] = c->cfg.het_fiducial[j];
  if (L.phase_marg) th[12] = 0.0;
  if (!(th[0] > 0.0) || !(th[1] > 0.0) || th[1] > 1.0 || !(th[6] > 0.0)) return fail(c, SWIG_E_ARG, "invalid fiducial theta");
  double* th_d = nullptr;
  double2* h_d = nullptr;
  std::vector<double2> h0((size_t)n_det * n);
  CUDA_TRY(c, cudaMalloc(&B.het_fid, sizeof(EvalRecord)));
  CUDA_TRY(c, cudaMalloc(&th_d, sizeof(th)));
  cudaError_t e = cudaMalloc(&h_d, sizeof(double2) * h0.size());
  if (e == cudaSuccess) e = cudaMemcpy(th_d, th, sizeof(th), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_waveform(L, th_d, B.het_fid, h_d, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMemcpy(h0.data(), h_d, sizeof(double2) * h0.size(), cudaMemcpyDeviceToHost);
  EvalRecord fid{};
  if (e == cudaSuccess) e = cudaMemcpy(&fid, B.het_fid, sizeof(EvalRecord), cudaMemcpyDeviceToHost);
  cudaFree(th_d);
  if (h_d) cudaFree(h_d);
  if (e != cudaSuccess) return fail(c, SWIG_E_CUDA, std::string("heterodyne fiducial: ") + cudaGetErrorString(e));
  c->n_launches += 2;
  c->d2h_bytes += sizeof(double2) * h0.size() + sizeof(EvalRecord);
  if (!fid.valid) return fail(c, SWIG_E_ARG, "invalid fiducial theta");
  for (int i = 0; i < n_det; ++i)
    if (!(fid.cre[i] * fid.cre[i] + fid.cim[i] * fid.cim[i] > 0.0))
      return fail(c, SWIG_E_ARG, "fiducial waveform vanishes in detector " + std::to_string(i));
  // summary data per detector and bin
  std::vector<float4> coef;
  std::vector<float2> coefB;
  std::vector<double> a01;  // FP64 (A0.re, A0.im, A1.re, A1.im) for the edge weights
  het_summary(f, idx, nb, n_det, c->df, c->data, c->psd, h0, coef, coefB, a01);
  std::vector<float> inv_w(nb);
  for (int b = 0; b < nb; ++b) inv_w[b] = (float)(1.0 / (f[idx[b + 1]] - f[idx[b]]));
  std::vector<float> eb((size_t)(nb + 1) * 2 * NBASIS), ef((size_t)(nb + 1) * 2);
  // transposed (row per basis function and hi/lo part) so that a warp reads
  // 32 consecutive edges of a row
  const size_t ne = (size_t)nb + 1;
  for (int q = 0; q <= nb; ++q) {
    const double fe = f[idx[q]];
    for (int j = 0; j < NBASIS; ++j) {
      const double v = (j == B_ONE) ? 1.0 : basis_derivative(kBasisPow[j], kBasisLog[j], 0, fe);
      split_df(v, &eb[2 * j * ne + q], &eb[(2 * j + 1) * ne + q]);
    }
    split_df(fe, &ef[q], &ef[ne + q]);
  }
  // chunk anchor tables (kernels.h HetChunkRow)
  std::vector<float> ct, dfe;
  const int nc = het_chunk_tables(f, idx, nb, ct, dfe);
  CUDA_TRY(c, cudaMalloc(&B.het_chunk, sizeof(float) * ct.size()));
  CUDA_TRY(c, cudaMalloc(&B.het_dfe, sizeof(float) * dfe.size()));
  CUDA_TRY(c, cudaMemcpy(B.het_chunk, ct.data(), sizeof(float) * ct.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(B.het_dfe, dfe.data(), sizeof(float) * dfe.size(), cudaMemcpyHostToDevice));
  c->h2d_bytes += sizeof(float) * (ct.size() + dfe.size());
  B.het_nc = nc;
  for (int i = 0; i < n_det; ++i) L.het_fid_iden[i] = 1.0 / (fid.cre[i] * fid.cre[i] + fid.cim[i] * fid.cim[i]);
  CUDA_TRY(c, cudaMalloc(&B.het_edge_basis, sizeof(float) * eb.size()));
  CUDA_TRY(c, cudaMalloc(&B.het_edge_f, sizeof(float) * ef.size()));
  CUDA_TRY(c, cudaMalloc(&B.het_inv_width, sizeof(float) * inv_w.size()));
  CUDA_TRY(c, cudaMalloc(&B.het_coef, sizeof(float4) * coef.size()));
  CUDA_TRY(c, cudaMalloc(&B.het_coefB, sizeof(float2) * coefB.size()));
  CUDA_TRY(c, cudaMemcpy(B.het_edge_basis, eb.data(), sizeof(float) * eb.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(B.het_edge_f, ef.data(), sizeof(float) * ef.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(B.het_inv_width, inv_w.data(), sizeof(float) * inv_w.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(B.het_coef, coef.data(), sizeof(float4) * coef.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(B.het_coefB, coefB.data(), sizeof(float2) * coefB.size(), cudaMemcpyHostToDevice));
  c->h2d_bytes += sizeof(float) * (eb.size() + ef.size() + inv_w.size()) + sizeof(float4) * coef.size() +
                  sizeof(float2) * coefB.size();
  if (L.tm_n > 0) {
    std::vector<float2> g, w;
    L.tm_M = 0;
    L.tm_pieces = L.tm_points = 0;
    std::vector<int> ptr, edge;
    std::vector<float> wt, corr;
    std::vector<float2> tw;
    if (L.tm_n >= kNufftMinNodes && L.tm_n <= kNufftMaxNodes) {
      std::vector<double> fe(nb + 1);
      for (int q = 0; q <= nb; ++q) fe[q] = f[idx[q]];
      het_nufft_tables(fe, L.tm_n, L.tm_dt, kNufftWidth, &L.tm_M, &L.tm_j0, ptr, edge, wt, corr, tw);
      L.tm_dref = L.tm_t0 + (double)L.tm_j0 * L.tm_dt;
      if (ptr.empty()) L.tm_M = 0;
    }
    // with the non-uniform FFT the edge weights carry the reference rotation,
    // so the bin pass stores c_e = y_e exp(-2 pi i f_e dt_ref) directly
    het_tm_tables(a01, f, idx, nb, n_det, L.tm_dt, g, w, L.tm_M > 0 ? L.tm_dref : 0.0);
    if (L.tm_M > 0) {
      // gather pieces: each grid point's entries in runs of at most
      // kNufftPiece (summed by one lane each), and the grid points with
      // entries (their pieces are combined in order)
      std::vector<int4> piece, point;
      nufft_pieces(ptr, edge, L.tm_M, piece, point);
      L.tm_pieces = (int)piece.size();
      L.tm_points = (int)point.size();
      CUDA_TRY(c, cudaMalloc(&B.het_nu_piece, sizeof(int4) * std::max<size_t>(1, piece.size())));
      CUDA_TRY(c, cudaMalloc(&B.het_nu_point, sizeof(int4) * std::max<size_t>(1, point.size())));
      if (!piece.empty()) {
        CUDA_TRY(c, cudaMemcpy(B.het_nu_piece, piece.data(), sizeof(int4) * piece.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(B.het_nu_point, point.data(), sizeof(int4) * point.size(), cudaMemcpyHostToDevice));
      }
      c->h2d_bytes += sizeof(int4) * (piece.size() + point.size());
      CUDA_TRY(c, cudaMalloc(&B.het_nu_wt, sizeof(float) * std::max<size_t>(1, wt.size())));
      CUDA_TRY(c, cudaMalloc(&B.het_nu_corr, sizeof(float) * corr.size()));
      tw = nufft_stage_twiddles(tw, L.tm_M);
      CUDA_TRY(c, cudaMalloc(&B.het_nu_tw, sizeof(float2) * tw.size()));
      CUDA_TRY(c, cudaMemcpy(B.het_nu_wt, wt.data(), sizeof(float) * wt.size(), cudaMemcpyHostToDevice));
      CUDA_TRY(c, cudaMemcpy(B.het_nu_corr, corr.data(), sizeof(float) * corr.size(), cudaMemcpyHostToDevice));
      CUDA_TRY(c, cudaMemcpy(B.het_nu_tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice));
      c->h2d_bytes += sizeof(float) * (wt.size() + corr.size()) + sizeof(float2) * tw.size();
    }
    CUDA_TRY(c, cudaMalloc(&B.het_tm_g, sizeof(float2) * g.size()));
    CUDA_TRY(c, cudaMalloc(&B.het_tm_w, sizeof(float2) * w.size()));
    CUDA_TRY(c, cudaMemcpy(B.het_tm_g, g.data(), sizeof(float2) * g.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(B.het_tm_w, w.data(), sizeof(float2) * w.size(), cudaMemcpyHostToDevice));
    c->h2d_bytes += sizeof(float2) * (g.size() + w.size());
  }
  B.het_nb = nb;
  return SWIG_OK;
}

int make_sky_frame(swig_ctx* c, SkyFrame* F) {
  std::memset(F, 0, sizeof(*F));
  if (c->sky_a < 0) return SWIG_OK;
  if (!c->det_set[c->sky_a] || !c->det_set[c->sky_b]) return fail(c, SWIG_E_STATE, "sky-frame detectors not set");
  const swig_param& az = c->params[9];
  const swig_param& zen = c->params[10];
  if (az.mode != SWIG_MODE_SAMPLE || zen.mode != SWIG_MODE_SAMPLE || az.kind != SWIG_PRIOR_UNIFORM ||
      zen.kind != SWIG_PRIOR_SINE || std::fabs(az.lo) > 1e-12 || std::fabs(az.hi - 2.0 * kPi) > 1e-9 ||
      std::fabs(zen.lo) > 1e-12 || std::fabs(zen.hi - kPi) > 1e-9 || az.block != zen.block)
    return fail(c, SWIG_E_ARG,
                "the detector sky frame needs slot 9 (azimuth) uniform on [0, 2 pi] and slot 10 (zenith) sine on "
                "[0, pi], both sampled in one block");
  double b[3], nb = 0.0;
  for (int k = 0; k < 3; ++k) {
    b[k] = c->vertex[c->sky_a][k] - c->vertex[c->sky_b][k];
    nb += b[k] * b[k];
  }
  nb = std::sqrt(nb);
  if (!(nb > 0.0)) return fail(c, SWIG_E_ARG, "the sky-frame detectors share a vertex");
  for (int k = 0; k < 3; ++k) F->ez[k] = b[k] / nb;
  // ex: the Earth's rotation axis made orthogonal to ez (or the x axis if parallel)
  double x[3] = {-F->ez[2] * F->ez[0], -F->ez[2] * F->ez[1], 1.0 - F->ez[2] * F->ez[2]};
  double nx = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  if (nx < 1e-12) {
    x[0] = 1.0 - F->ez[0] * F->ez[0];
    x[1] = -F->ez[0] * F->ez[1];
    x[2] = -F->ez[0] * F->ez[2];
    nx = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  }
  for (int k = 0; k < 3; ++k) F->ex[k] = x[k] / nx;
  F->ey[0] = F->ez[1] * F->ex[2] - F->ez[2] * F->ex[1];
  F->ey[1] = F->ez[2] * F->ex[0] - F->ez[0] * F->ex[2];
  F->ey[2] = F->ez[0] * F->ex[1] - F->ez[1] * F->ex[0];
  F->gmst = c->gmst;
  F->on = 1;
  return SWIG_OK;
}

int ensure_scratch(swig_ctx* c, int n) {
  DeviceBuffers& B = c->B;
  if (n <= B.cap) return SWIG_OK;
  free_scratch(B);
  const int cap = std::max(n, 256);
  const size_t ntiles = std::max(c->L.n_tiles, 1);
  CUDA_TRY(c, cudaMalloc(&B.rec, sizeof(EvalRecord) * cap));
  CUDA_TRY(c, cudaMalloc(&B.anchors, sizeof(float) * kAnchorStride * ntiles * cap));
  const size_t units = (size_t)c->L.n_slices * 4;  // up to 4 work units per (theta, slice)
  CUDA_TRY(c, cudaMalloc(&B.partials32, sizeof(float) * kPartialStride * units * cap));
  CUDA_TRY(c, cudaMalloc(&B.partials64, sizeof(double) * kPartialStride * units * cap));
  CUDA_TRY(c, cudaMalloc(&B.theta, sizeof(double) * SWIG_N_PARAMS * cap));
  CUDA_TRY(c, cudaMalloc(&B.out, sizeof(double) * cap));
  CUDA_TRY(c, cudaMalloc(&B.u, sizeof(double) * SWIG_N_PARAMS * cap));
  B.cap = cap;
  return SWIG_OK;
}

int current_precision(const swig_ctx* c) { return c->cfg_set ? c->cfg.precision : SWIG_PREC_MIXED; }

// Slices: contiguous whole 32-bin chunks, one CTA each, cut at equal
// estimated cost.  With a tile plan (mixed precision) every tile of more than
// 32 bins adds about one chunk's cost (its anchor, and every lane's crossing
// into it in the bin loop), and a chunk holding tiles of 32 bins or fewer
// (every lane crosses into a new tile on every step) costs about 2.3 chunks,
// as measured on GB300 with the per-CTA sweep counters of the persistent
// sampler.  Up to sm_count slices (more if one slice's data would not fit in
// shared memory).
void plan_slices(int64_t n, int n_det, int sm_count, const std::vector<TileInfo>& tiles,
                 std::vector<int>& slice_begin, int* max_bins_out) {
  const int n_chunks = (int)((n + kChunk - 1) / kChunk);
  std::vector<double> chunk_cost(n_chunks, 1.0);
  for (const TileInfo& ti : tiles) {
    double& cc = chunk_cost[ti.k0 / kChunk];
    cc = ti.nbins <= kChunk ? std::max(cc, 2.33) : cc + 1.0;
  }
  double total_cost = 0.0;
  for (double v : chunk_cost) total_cost += v;
  int n_slices = std::min(sm_count, std::max(1, n_chunks / 4));
  const size_t smem_cap = 200 * 1024;
  int max_bins = 0;
  for (;;) {
    slice_begin.assign(1, 0);
    double acc = 0.0;
    int s = 1;
    for (int ch = 0; ch < n_chunks && s < n_slices; ++ch) {
      acc += chunk_cost[ch];
      if (acc >= total_cost * s / n_slices && ch + 1 < n_chunks) {
        slice_begin.push_back((ch + 1) * kChunk);
        ++s;
      }
    }
    slice_begin.push_back((int)n);
    max_bins = 0;
    for (size_t q = 0; q + 1 < slice_begin.size(); ++q) max_bins = std::max(max_bins, slice_begin[q + 1] - slice_begin[q]);
    if (sweep_smem_bytes(n_det, max_bins) <= smem_cap || n_slices >= n_chunks) break;
    n_slices = std::min(n_chunks, n_slices * 2);
  }
  *max_bins_out = max_bins;
}

// Validate the problem and (re)build every device-side table.
int prepare(swig_ctx* c) {
  if (!c->dirty) return SWIG_OK;
  if (!c->grid_set) return fail(c, SWIG_E_STATE, "grid not set");
  int n_det = 0;
  while (n_det < SWIG_MAX_DET && c->det_set[n_det]) ++n_det;
  if (n_det == 0) return fail(c, SWIG_E_STATE, "no detector set");
  for (int i = n_det; i < SWIG_MAX_DET; ++i)
    if (c->det_set[i]) return fail(c, SWIG_E_STATE, "detectors must be set contiguously from index 0");
  const int64_t n = c->n_bins;
  for (int i = 0; i < n_det; ++i) {
    if ((int64_t)c->data[i].size() != 2 * n) return fail(c, SWIG_E_STATE, "data of detector " + std::to_string(i) + " not set for this grid");
    if ((int64_t)c->psd[i].size() != n) return fail(c, SWIG_E_STATE, "psd of detector " + std::to_string(i) + " not set for this grid");
  }
  CUDA_TRY(c, cudaSetDevice(c->device));
  free_problem(c->B);
  free_scratch(c->B);

  LikeConst& L = c->L;
  std::memset(&L, 0, sizeof(L));
  L.n_det = n_det;
  L.n_bins = (int)n;
  L.k_min = (int)c->k_min;
  L.df = c->df;
  L.gmst = c->gmst;
  L.phase_marg = c->prior_set && c->params[12].mode == SWIG_MODE_MARG;
  L.dist_marg = c->prior_set && c->params[6].mode == SWIG_MODE_MARG;
  if (L.dist_marg) {
    L.d_kind = c->params[6].kind;
    L.d_lo = c->params[6].lo;
    L.d_hi = c->params[6].hi;
    gauss_legendre(kGaussLegendre, L.gl_x, L.gl_w);
  }
  if (L.dist_marg && c->cfg_set && c->cfg.likelihood == SWIG_LIKE_HET)
    return fail(c, SWIG_E_ARG, "distance marginalisation is implemented for the full-grid likelihood only");
  if (c->prior_set && c->params[11].mode == SWIG_MODE_MARG) {
    // time marginalisation: midpoint grid over the uniform t_c prior, templates
    // at the fiducial's t_c shifted to each node (heterodyned bins only)
    if (!c->cfg_set || c->cfg.likelihood != SWIG_LIKE_HET)
      return fail(c, SWIG_E_ARG, "time marginalisation is implemented for the heterodyned likelihood only");
    if (c->cfg.tmarg_nodes < 1) return fail(c, SWIG_E_ARG, "time marginalisation needs tmarg_nodes >= 1");
    if (c->cfg.het_bins > kMaxTmBins) return fail(c, SWIG_E_ARG, "time marginalisation supports at most 16384 heterodyned bins");
    if (!std::isfinite(c->cfg.het_fiducial[11])) return fail(c, SWIG_E_ARG, "non-finite fiducial t_c");
    const swig_param& p = c->params[11];
    c->params[11].value = c->cfg.het_fiducial[11];
    L.tm_n = c->cfg.tmarg_nodes;
    L.tm_lo = p.lo;
    L.tm_dt = (p.hi - p.lo) / L.tm_n;
    L.tm_tref = c->cfg.het_fiducial[11];
    L.tm_t0 = L.tm_lo + 0.5 * L.tm_dt - L.tm_tref;
  }
  const int prec = current_precision(c);
  L.fast_epilogue = prec == SWIG_PREC_MIXED ? 1 : 0;

  // D_i(k) = 4 df conj(d_i) f^-7/6 / S_i,  K_i = 4 df sum f^-7/3 / S_i,  <d|d>
  std::vector<double> dre, dim;
  double dmax[SWIG_MAX_DET], dd_sum = 0.0;
  weight_data(c, n_det, dre, dim, L.K, &dd_sum, dmax);
  for (int i = 0; i < n_det; ++i) {
    L.inv_scale[i] = prec == SWIG_PREC_MIXED ? (dmax[i] > 0.0 ? dmax[i] : 1.0) : 1.0;
    for (int r = 0; r < 3; ++r) L.vertex[i][r] = c->vertex[i][r];
    const double* x = c->xarm[i];
    const double* y = c->yarm[i];
    L.dten[i][0] = 0.5 * (x[0] * x[0] - y[0] * y[0]);
    L.dten[i][1] = 0.5 * (x[0] * x[1] - y[0] * y[1]);
    L.dten[i][2] = 0.5 * (x[0] * x[2] - y[0] * y[2]);
    L.dten[i][3] = 0.5 * (x[1] * x[1] - y[1] * y[1]);
    L.dten[i][4] = 0.5 * (x[1] * x[2] - y[1] * y[2]);
    L.dten[i][5] = 0.5 * (x[2] * x[2] - y[2] * y[2]);
  }
  L.DD = dd_sum;
  {
    const double a1 = std::sqrt(5.0 / 24.0) * std::pow(kPi, -2.0 / 3.0) * std::pow(kMtsunS, 5.0 / 6.0) * kCSI / kMpcM;
    for (int i = 0; i < n_det; ++i) {
      L.amp_s[i] = (float)(L.inv_scale[i] * a1);
      L.amp_k[i] = (float)(L.K[i] * a1 * a1);
      L.amp1 = a1;
    }
  }

  std::vector<TileInfo> tiles;
  std::vector<TileBasis> basis;
  if (prec == SWIG_PREC_MIXED) plan_tiles(c, tiles, basis);
  std::vector<int> slice_begin;
  int max_bins = 0;
  plan_slices(n, n_det, c->sm_count, tiles, slice_begin, &max_bins);
  int n_slices = (int)slice_begin.size() - 1;
  L.n_slices = n_slices;
  c->B.max_slice_bins = max_bins;

  DeviceBuffers& B = c->B;
  CUDA_TRY(c, cudaMalloc(&B.slice_begin, sizeof(int) * (n_slices + 1)));
  CUDA_TRY(c, cudaMemcpy(B.slice_begin, slice_begin.data(), sizeof(int) * (n_slices + 1), cudaMemcpyHostToDevice));
  c->h2d_bytes += sizeof(int) * (n_slices + 1);

  if (prec == SWIG_PREC_MIXED) {
    std::vector<float2> d32((size_t)n_det * n);
    for (int i = 0; i < n_det; ++i) {
      const double s = 1.0 / L.inv_scale[i];
      for (int64_t k = 0; k < n; ++k) d32[i * n + k] = make_float2((float)(dre[i * n + k] * s), (float)(dim[i * n + k] * s));
    }
    CUDA_TRY(c, cudaMalloc(&B.data32, sizeof(float2) * d32.size()));
    CUDA_TRY(c, cudaMemcpy(B.data32, d32.data(), sizeof(float2) * d32.size(), cudaMemcpyHostToDevice));
    c->h2d_bytes += sizeof(float2) * d32.size() + sizeof(TileInfo) * tiles.size() + sizeof(TileBasis) * basis.size() +
                    sizeof(int) * n;
    L.n_tiles = (int)tiles.size();
    std::vector<int> bin_tile(n);
    for (int t = 0; t < L.n_tiles; ++t)
      for (int k = tiles[t].k0; k < tiles[t].k0 + tiles[t].nbins; ++k) bin_tile[k] = t;
    CUDA_TRY(c, cudaMalloc(&B.tiles, sizeof(TileInfo) * tiles.size()));
    CUDA_TRY(c, cudaMemcpy(B.tiles, tiles.data(), sizeof(TileInfo) * tiles.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMalloc(&B.basis, sizeof(TileBasis) * basis.size()));
    CUDA_TRY(c, cudaMemcpy(B.basis, basis.data(), sizeof(TileBasis) * basis.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMalloc(&B.bin_tile, sizeof(int) * n));
    CUDA_TRY(c, cudaMemcpy(B.bin_tile, bin_tile.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    CUDA_TRY(c, set_sweep_smem_limit(sweep_smem_bytes(n_det, max_bins)));
  } else {
    std::vector<double2> d64((size_t)n_det * n);
    for (size_t k = 0; k < d64.size(); ++k) d64[k] = make_double2(dre[k], dim[k]);
    CUDA_TRY(c, cudaMalloc(&B.data64, sizeof(double2) * d64.size()));
    CUDA_TRY(c, cudaMemcpy(B.data64, d64.data(), sizeof(double2) * d64.size(), cudaMemcpyHostToDevice));
    c->h2d_bytes += sizeof(double2) * d64.size() + sizeof(double) * 3 * n;
    std::vector<double> ftab((size_t)3 * n);
    for (int64_t k = 0; k < n; ++k) {
      const double f = (double)(c->k_min + k) * c->df;
      ftab[3 * k] = 1.0 / std::cbrt(f);
      ftab[3 * k + 1] = std::cbrt(f);
      ftab[3 * k + 2] = std::log(f);
    }
    CUDA_TRY(c, cudaMalloc(&B.ftab, sizeof(double) * ftab.size()));
    CUDA_TRY(c, cudaMemcpy(B.ftab, ftab.data(), sizeof(double) * ftab.size(), cudaMemcpyHostToDevice));
    L.n_tiles = 0;
  }
  // sweep pieces: whole 32-bin chunks, at most 8 chunks and 32 tiles each, so
  // that a warp computes a piece's anchors with one lane per tile
  {
    std::vector<int> bt;
    if (prec == SWIG_PREC_MIXED) {
      bt.resize(n);
      CUDA_TRY(c, cudaMemcpy(bt.data(), B.bin_tile, sizeof(int) * n, cudaMemcpyDeviceToHost));
    }
    std::vector<int> pb, sp(n_slices + 1);
    int maxp = 1;
    for (int s = 0; s < n_slices; ++s) {
      sp[s] = (int)pb.size();
      int b = slice_begin[s];
      while (b < slice_begin[s + 1]) {
        pb.push_back(b);
        int e = std::min<int>(b + kChunk, slice_begin[s + 1]);
        while (e < slice_begin[s + 1] && e - b < 8 * kChunk) {
          const int e2 = std::min<int>(e + kChunk, slice_begin[s + 1]);
          if (!bt.empty() && bt[e2 - 1] - bt[b] + 1 > 32) break;
          e = e2;
        }
        b = e;
      }
      pb.push_back(slice_begin[s + 1]);
      maxp = std::max(maxp, (int)pb.size() - sp[s] - 1);
    }
    sp[n_slices] = (int)pb.size();
    B.n_pieces = (int)pb.size() - n_slices;
    B.max_pieces = maxp;
    CUDA_TRY(c, cudaMalloc(&B.piece_begin, sizeof(int) * pb.size()));
    CUDA_TRY(c, cudaMemcpy(B.piece_begin, pb.data(), sizeof(int) * pb.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMalloc(&B.slice_piece, sizeof(int) * sp.size()));
    CUDA_TRY(c, cudaMemcpy(B.slice_piece, sp.data(), sizeof(int) * sp.size(), cudaMemcpyHostToDevice));
  }
  // prior slots (defaults when no prior was set: every slot sampled uniform on [0,1])
  PriorSlot slots[SWIG_N_PARAMS];
  for (int i = 0; i < SWIG_N_PARAMS; ++i) {
    const swig_param& p = c->params[i];
    slots[i] = c->prior_set ? make_prior_slot(p.kind, p.mode, p.lo, p.hi, p.value) : make_prior_slot(0, 0, 0.0, 1.0, 0.0);
  }
  CUDA_TRY(c, cudaMalloc(&B.prior, sizeof(slots)));
  CUDA_TRY(c, cudaMemcpy(B.prior, slots, sizeof(slots), cudaMemcpyHostToDevice));
  c->prepared_precision = prec;
  c->prepared_like = c->cfg_set ? c->cfg.likelihood : SWIG_LIKE_FULL;
  if (c->prepared_like == SWIG_LIKE_HET) {
    const int rc = prepare_het(c);
    if (rc) return rc;
  }
  c->dirty = false;
  return SWIG_OK;
}

int loglike_device(swig_ctx* c, const double* theta_dev, int64_t n, double* out_dev, cudaStream_t st) {
  const int chunk = 4096;
  for (int64_t off = 0; off < n; off += chunk) {
    const int m = (int)std::min<int64_t>(chunk, n - off);
    int rc = ensure_scratch(c, m);
    if (rc) return rc;
    cudaError_t e;
    if (c->prepared_like == SWIG_LIKE_HET) {
      e = launch_loglike_het(c->L, c->B, theta_dev + off * SWIG_N_PARAMS, m, out_dev + off, st);
      c->n_launches += 2;
    } else {
      e = c->prepared_precision == SWIG_PREC_MIXED
              ? launch_loglike_mixed(c->L, c->B, theta_dev + off * SWIG_N_PARAMS, m, out_dev + off, st)
              : launch_loglike_fp64(c->L, c->B, theta_dev + off * SWIG_N_PARAMS, m, out_dev + off, st);
      c->n_launches += c->prepared_precision == SWIG_PREC_MIXED ? 4 : 3;
    }
    if (e != cudaSuccess) return fail(c, SWIG_E_CUDA, std::string("likelihood launch: ") + cudaGetErrorString(e));
  }
  return SWIG_OK;
}

}  // namespace swig

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

int swig_create(swig_ctx** out, int cuda_device) {
  if (!out) {
    g_create_error = "null output pointer";
    return SWIG_E_ARG;
  }
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) {
    g_create_error = std::string("cudaGetDeviceCount: ") + cudaGetErrorString(e);
    return SWIG_E_CUDA;
  }
  if (cuda_device < 0 || cuda_device >= count) {
    g_create_error = "device index out of range";
    return SWIG_E_ARG;
  }
  swig_ctx* c = new (std::nothrow) swig_ctx();
  if (!c) {
    g_create_error = "out of host memory";
    return SWIG_E_NOMEM;
  }
  c->device = cuda_device;
  e = cudaSetDevice(cuda_device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, cuda_device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    g_create_error = std::string("device setup: ") + cudaGetErrorString(e);
    delete c;
    return SWIG_E_CUDA;
  }
  *out = c;
  return SWIG_OK;
}

void swig_destroy(swig_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  swig_sampler_release(c);
  swig_mlp_release(c);
  free_problem(c->B);
  free_scratch(c->B);
  if (c->stream && c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* swig_last_error(const swig_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int swig_set_grid(swig_ctx* c, double f_min, double f_max, double df) {
  if (!c) return SWIG_E_ARG;
  if (!(f_min > 0.0) || !(f_max > f_min) || !(df > 0.0) || !std::isfinite(f_max))
    return fail(c, SWIG_E_ARG, "grid needs 0 < f_min < f_max and df > 0");
  const double k0 = std::ceil(f_min / df - 1e-9), k1 = std::floor(f_max / df + 1e-9);
  if (k1 < k0 || k1 - k0 + 1 > (double)(1 << 22)) return fail(c, SWIG_E_ARG, "grid must have 1 .. 2^22 bins");
  c->f_min = f_min;
  c->f_max = f_max;
  c->df = df;
  c->k_min = (int64_t)k0;
  c->n_bins = (int64_t)(k1 - k0) + 1;
  c->grid_set = true;
  for (int i = 0; i < SWIG_MAX_DET; ++i) {
    c->data[i].clear();
    c->psd[i].clear();
  }
  c->dirty = true;
  return SWIG_OK;
}

int swig_set_detector(swig_ctx* c, int idx, const double vertex_m[3], const double x_arm[3], const double y_arm[3]) {
  if (!c) return SWIG_E_ARG;
  if (idx < 0 || idx >= SWIG_MAX_DET || !vertex_m || !x_arm || !y_arm) return fail(c, SWIG_E_ARG, "bad detector index or null vector");
  for (int r = 0; r < 3; ++r)
    if (!std::isfinite(vertex_m[r]) || !std::isfinite(x_arm[r]) || !std::isfinite(y_arm[r]))
      return fail(c, SWIG_E_NUMERIC, "non-finite detector geometry");
  for (int r = 0; r < 3; ++r) {
    c->vertex[idx][r] = vertex_m[r];
    c->xarm[idx][r] = x_arm[r];
    c->yarm[idx][r] = y_arm[r];
  }
  c->det_set[idx] = true;
  c->dirty = true;
  return SWIG_OK;
}

int swig_set_time_ref(swig_ctx* c, double gmst_rad) {
  if (!c) return SWIG_E_ARG;
  if (!std::isfinite(gmst_rad)) return fail(c, SWIG_E_NUMERIC, "non-finite GMST");
  c->gmst = gmst_rad;
  c->dirty = true;
  return SWIG_OK;
}

int swig_set_data(swig_ctx* c, int det, const double* re_im, int64_t n) {
  if (!c) return SWIG_E_ARG;
  if (!c->grid_set) return fail(c, SWIG_E_STATE, "set the grid before data");
  if (det < 0 || det >= SWIG_MAX_DET || !re_im) return fail(c, SWIG_E_ARG, "bad detector index or null data");
  if (n != c->n_bins) return fail(c, SWIG_E_ARG, "data length must equal the number of grid bins");
  for (int64_t k = 0; k < 2 * n; ++k)
    if (!std::isfinite(re_im[k])) return fail(c, SWIG_E_NUMERIC, "non-finite data value");
  c->data[det].assign(re_im, re_im + 2 * n);
  c->dirty = true;
  return SWIG_OK;
}

int swig_set_psd(swig_ctx* c, int det, const double* psd, int64_t n) {
  if (!c) return SWIG_E_ARG;
  if (!c->grid_set) return fail(c, SWIG_E_STATE, "set the grid before the PSD");
  if (det < 0 || det >= SWIG_MAX_DET || !psd) return fail(c, SWIG_E_ARG, "bad detector index or null psd");
  if (n != c->n_bins) return fail(c, SWIG_E_ARG, "psd length must equal the number of grid bins");
  for (int64_t k = 0; k < n; ++k)
    if (!std::isfinite(psd[k]) || !(psd[k] > 0.0)) return fail(c, SWIG_E_NUMERIC, "PSD values must be finite and > 0");
  c->psd[det].assign(psd, psd + n);
  c->dirty = true;
  return SWIG_OK;
}

int swig_set_prior(swig_ctx* c, const swig_param* params, int n_params) {
  if (!c) return SWIG_E_ARG;
  if (!params || n_params != SWIG_N_PARAMS) return fail(c, SWIG_E_ARG, "prior needs exactly 13 slots");
  int n_sampled = 0;
  for (int i = 0; i < SWIG_N_PARAMS; ++i) {
    const swig_param& p = params[i];
    if (p.mode < 0 || p.mode > 2 || p.kind < 0 || p.kind > 3) return fail(c, SWIG_E_ARG, "bad prior kind or mode in slot " + std::to_string(i));
    if (p.mode == SWIG_MODE_MARG && i != 12 && i != 6 && i != 11)
      return fail(c, SWIG_E_ARG, "only d_L (slot 6), t_c (slot 11) and phi_c (slot 12) can be marginalised");
    if (p.mode == SWIG_MODE_MARG && i == 11 &&
        (p.kind != SWIG_PRIOR_UNIFORM || !std::isfinite(p.lo) || !std::isfinite(p.hi) || !(p.hi > p.lo)))
      return fail(c, SWIG_E_ARG, "a marginalised t_c needs a uniform prior with lo < hi");
    if (p.mode == SWIG_MODE_MARG && i == 6 &&
        (!(p.lo > 0.0) || !(p.hi > p.lo) || !std::isfinite(p.hi) ||
         (p.kind != SWIG_PRIOR_UNIFORM && p.kind != SWIG_PRIOR_POWER2)))
      return fail(c, SWIG_E_ARG, "a marginalised d_L needs a uniform or power-law-2 prior on 0 < lo < hi");
    if (p.mode == SWIG_MODE_SAMPLE) {
      if (!std::isfinite(p.lo) || !std::isfinite(p.hi) || !(p.hi > p.lo)) return fail(c, SWIG_E_ARG, "sampled slot " + std::to_string(i) + " needs lo < hi");
      if (p.block < 0 || p.block >= 16) return fail(c, SWIG_E_ARG, "block id must be in [0, 16)");
      ++n_sampled;
    }
    if (p.mode == SWIG_MODE_FIXED && !std::isfinite(p.value)) return fail(c, SWIG_E_NUMERIC, "non-finite fixed value");
  }
  if (n_sampled == 0) return fail(c, SWIG_E_ARG, "at least one parameter must be sampled");
  std::memcpy(c->params, params, sizeof(swig_param) * SWIG_N_PARAMS);
  // a marginalised slot is evaluated at a fixed value: phi_c = 0, d_L = 1 Mpc
  if (c->params[12].mode == SWIG_MODE_MARG) c->params[12].value = 0.0;
  if (c->params[6].mode == SWIG_MODE_MARG) c->params[6].value = 1.0;
  // t_c marginalised: templates at the heterodyne fiducial's t_c
  if (c->params[11].mode == SWIG_MODE_MARG) c->params[11].value = c->cfg_set ? c->cfg.het_fiducial[11] : 0.0;
  c->prior_set = true;
  c->n_sampled = n_sampled;
  c->dirty = true;
  return SWIG_OK;
}

int swig_set_sampler(swig_ctx* c, const swig_sampler_cfg* cfg) {
  if (!c) return SWIG_E_ARG;
  if (!cfg) return fail(c, SWIG_E_ARG, "null sampler configuration");
  if (cfg->nlive < 2 || cfg->nrep < 1 || cfg->nrep >= cfg->nlive) return fail(c, SWIG_E_ARG, "need nlive > nrep >= 1");
  if (cfg->nlive > (1 << 16)) return fail(c, SWIG_E_ARG, "nlive must be <= 65536");
  if (cfg->sweeps < 1 || cfg->steps_per_dim < 1) return fail(c, SWIG_E_ARG, "sweeps and steps_per_dim must be >= 1");
  if (cfg->precision != SWIG_PREC_FP64 && cfg->precision != SWIG_PREC_MIXED) return fail(c, SWIG_E_ARG, "bad precision");
  if (cfg->likelihood != SWIG_LIKE_FULL && cfg->likelihood != SWIG_LIKE_HET) return fail(c, SWIG_E_ARG, "bad likelihood");
  if (cfg->proposal != SWIG_PROPOSAL_COV && cfg->proposal != SWIG_PROPOSAL_LEARNED) return fail(c, SWIG_E_ARG, "bad proposal");
  if (cfg->likelihood == SWIG_LIKE_HET && (cfg->het_bins < 2 || cfg->het_bins > 65536)) return fail(c, SWIG_E_ARG, "het_bins must be in [2, 65536]");
  if (cfg->het_spacing != 0 && cfg->het_spacing != 1) return fail(c, SWIG_E_ARG, "het_spacing must be 0 or 1");
  if (!(cfg->dlogz < 0.0) || cfg->max_iter < 1) return fail(c, SWIG_E_ARG, "need dlogz < 0 and max_iter >= 1");
  if (cfg->tmarg_nodes < 0 || cfg->tmarg_nodes > kMaxTmNodes) return fail(c, SWIG_E_ARG, "tmarg_nodes must be in [0, 65536]");
  if (cfg->cache_off != 0 && cfg->cache_off != 1) return fail(c, SWIG_E_ARG, "cache_off must be 0 or 1");
  if (cfg->flow_parts < 0 || cfg->flow_parts > 4) return fail(c, SWIG_E_ARG, "flow_parts must be 0..4");
  if (cfg->stepout_one_end != 0 && cfg->stepout_one_end != 1)
    return fail(c, SWIG_E_ARG, "stepout_one_end must be 0 or 1");
  if (c->cfg_set && (c->cfg.precision != cfg->precision || c->cfg.likelihood != cfg->likelihood ||
                     c->cfg.het_bins != cfg->het_bins || c->cfg.het_spacing != cfg->het_spacing ||
                     c->cfg.tmarg_nodes != cfg->tmarg_nodes ||
                     std::memcmp(c->cfg.het_fiducial, cfg->het_fiducial, sizeof(cfg->het_fiducial)) != 0))
    c->dirty = true;
  if (!c->cfg_set) c->dirty = true;
  c->cfg = *cfg;
  c->cfg_set = true;
  if (c->prior_set && c->params[11].mode == SWIG_MODE_MARG) c->params[11].value = cfg->het_fiducial[11];
  return SWIG_OK;
}

int swig_loglike_batch(swig_ctx* c, const double* theta, int64_t n, double* out_logl) {
  if (!c) return SWIG_E_ARG;
  if (n == 0) return SWIG_OK;
  if (n < 0 || n > (1 << 20) || !theta || !out_logl) return fail(c, SWIG_E_ARG, "need 0 <= n <= 2^20 and non-null buffers");
  int rc = prepare(c);
  if (rc) return rc;
  const int chunk = 4096;
  for (int64_t off = 0; off < n; off += chunk) {
    const int m = (int)std::min<int64_t>(chunk, n - off);
    if ((rc = ensure_scratch(c, m))) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->B.theta, theta + off * SWIG_N_PARAMS, sizeof(double) * SWIG_N_PARAMS * m, cudaMemcpyHostToDevice, c->stream));
    if ((rc = loglike_device(c, c->B.theta, m, c->B.out, c->stream))) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(out_logl + off, c->B.out, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  return SWIG_OK;
}

int swig_loglike_batch_dev(swig_ctx* c, const double* theta_dev, int64_t n, double* out_dev, void* stream) {
  if (!c) return SWIG_E_ARG;
  if (n == 0) return SWIG_OK;
  if (n < 0 || n > (1 << 20) || !theta_dev || !out_dev) return fail(c, SWIG_E_ARG, "need 0 <= n <= 2^20 and non-null buffers");
  int rc = prepare(c);
  if (rc) return rc;
  return loglike_device(c, theta_dev, n, out_dev, (cudaStream_t)stream);
}

int swig_inject(swig_ctx* c, const double* theta, double target_snr, const double* noise_re_im, double* out_re_im,
                double* theta_out) {
  if (!c) return SWIG_E_ARG;
  if (!theta || !out_re_im) return fail(c, SWIG_E_ARG, "null theta or output");
  if (!c->grid_set) return fail(c, SWIG_E_STATE, "grid not set");
  int n_det = 0;
  while (n_det < SWIG_MAX_DET && c->det_set[n_det]) ++n_det;
  if (n_det == 0) return fail(c, SWIG_E_STATE, "no detector set");
  const int64_t n = c->n_bins;
  if (target_snr > 0.0)
    for (int i = 0; i < n_det; ++i)
      if ((int64_t)c->psd[i].size() != n) return fail(c, SWIG_E_STATE, "PSDs are needed to scale to a target SNR");
  double th[SWIG_N_PARAMS];
  for (int j = 0; j < SWIG_N_PARAMS; ++j) th[j] = theta[j];
  if (!(th[0] > 0.0) || !(th[1] > 0.0) || th[1] > 1.0 || !(th[6] > 0.0)) return fail(c, SWIG_E_ARG, "invalid theta");
  CUDA_TRY(c, cudaSetDevice(c->device));
  LikeConst L;
  std::memset(&L, 0, sizeof(L));
  L.n_det = n_det;
  L.n_bins = (int)n;
  L.k_min = (int)c->k_min;
  L.df = c->df;
  L.gmst = c->gmst;
  L.phase_marg = 0;
  for (int i = 0; i < n_det; ++i) {
    for (int r = 0; r < 3; ++r) L.vertex[i][r] = c->vertex[i][r];
    const double* x = c->xarm[i];
    const double* y = c->yarm[i];
    L.dten[i][0] = 0.5 * (x[0] * x[0] - y[0] * y[0]);
    L.dten[i][1] = 0.5 * (x[0] * x[1] - y[0] * y[1]);
    L.dten[i][2] = 0.5 * (x[0] * x[2] - y[0] * y[2]);
    L.dten[i][3] = 0.5 * (x[1] * x[1] - y[1] * y[1]);
    L.dten[i][4] = 0.5 * (x[1] * x[2] - y[1] * y[2]);
    L.dten[i][5] = 0.5 * (x[2] * x[2] - y[2] * y[2]);
    if (target_snr > 0.0) {
      NSum K;
      for (int64_t k = 0; k < n; ++k) {
        const double f = (double)(c->k_min + k) * c->df;
        K.add(4.0 * c->df / c->psd[i][k] * std::pow(f, -7.0 / 3.0));
      }
      L.K[i] = K.value();
    }
  }
  double* th_d = nullptr;
  EvalRecord* rec_d = nullptr;
  double2* h_d = nullptr;
  std::vector<double2> h((size_t)n_det * n);
  EvalRecord rec;
  auto run = [&]() -> cudaError_t {
    cudaError_t e;
    if ((e = cudaMalloc(&th_d, sizeof(th)))) return e;
    if ((e = cudaMalloc(&rec_d, sizeof(EvalRecord)))) return e;
    if ((e = cudaMalloc(&h_d, sizeof(double2) * h.size()))) return e;
    for (int pass = 0; pass < 2; ++pass) {
      if ((e = cudaMemcpy(th_d, th, sizeof(th), cudaMemcpyHostToDevice))) return e;
      if ((e = launch_waveform(L, th_d, rec_d, h_d, c->stream))) return e;
      if ((e = cudaStreamSynchronize(c->stream))) return e;
      if ((e = cudaMemcpy(&rec, rec_d, sizeof(rec), cudaMemcpyDeviceToHost))) return e;
      if (pass == 0 && target_snr > 0.0) {
        double snr2 = 0.0;
        for (int i = 0; i < n_det; ++i) snr2 += (rec.cre[i] * rec.cre[i] + rec.cim[i] * rec.cim[i]) * L.K[i];
        th[6] *= std::sqrt(snr2) / target_snr;  // SNR scales as 1 / d_L
        continue;
      }
      break;
    }
    return cudaMemcpy(h.data(), h_d, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost);
  };
  const cudaError_t e = run();
  if (th_d) cudaFree(th_d);
  if (rec_d) cudaFree(rec_d);
  if (h_d) cudaFree(h_d);
  if (e != cudaSuccess) return fail(c, SWIG_E_CUDA, std::string("injection: ") + cudaGetErrorString(e));
  for (size_t k = 0; k < h.size(); ++k) {
    out_re_im[2 * k] = h[k].x + (noise_re_im ? noise_re_im[2 * k] : 0.0);
    out_re_im[2 * k + 1] = h[k].y + (noise_re_im ? noise_re_im[2 * k + 1] : 0.0);
  }
  if (theta_out)
    for (int j = 0; j < SWIG_N_PARAMS; ++j) theta_out[j] = th[j];
  return SWIG_OK;
}

int swig_set_stream(swig_ctx* c, void* stream) {
  if (!c) return SWIG_E_ARG;
  CUDA_TRY(c, cudaSetDevice(c->device));
  if (c->stream && c->own_stream) CUDA_TRY(c, cudaStreamDestroy(c->stream));
  if (stream) {
    c->stream = (cudaStream_t)stream;
    c->own_stream = false;
  } else {
    CUDA_TRY(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  return SWIG_OK;
}

int swig_set_sky_frame(swig_ctx* c, int det_a, int det_b) {
  if (!c) return SWIG_E_ARG;
  if (det_a < 0 && det_b < 0) {
    c->sky_a = c->sky_b = -1;
    return SWIG_OK;
  }
  if (det_a < 0 || det_b < 0 || det_a >= SWIG_MAX_DET || det_b >= SWIG_MAX_DET || det_a == det_b)
    return fail(c, SWIG_E_ARG, "need two different detector indices (or -1, -1 for the equatorial frame)");
  c->sky_a = det_a;
  c->sky_b = det_b;
  return SWIG_OK;
}

int swig_prior_transform(swig_ctx* c, const double* u, int64_t n, double* theta) {
  if (!c) return SWIG_E_ARG;
  if (!c->prior_set) return fail(c, SWIG_E_STATE, "prior not set");
  if (n == 0) return SWIG_OK;
  if (n < 0 || n > (1 << 20) || !u || !theta) return fail(c, SWIG_E_ARG, "need 0 <= n <= 2^20 and non-null buffers");
  CUDA_TRY(c, cudaSetDevice(c->device));
  const int ns = c->n_sampled;
  SkyFrame sky;
  const int rc = make_sky_frame(c, &sky);
  if (rc) return rc;
  PriorSlot slots[SWIG_N_PARAMS];
  for (int i = 0; i < SWIG_N_PARAMS; ++i) {
    const swig_param& p = c->params[i];
    slots[i] = make_prior_slot(p.kind, p.mode, p.lo, p.hi, p.value);
  }
  PriorSlot* slots_d = nullptr;
  double *u_d = nullptr, *th_d = nullptr;
  auto run = [&]() -> cudaError_t {
    cudaError_t e;
    if ((e = cudaMalloc(&slots_d, sizeof(slots)))) return e;
    if ((e = cudaMalloc(&u_d, sizeof(double) * ns * n))) return e;
    if ((e = cudaMalloc(&th_d, sizeof(double) * SWIG_N_PARAMS * n))) return e;
    if ((e = cudaMemcpyAsync(slots_d, slots, sizeof(slots), cudaMemcpyHostToDevice, c->stream))) return e;
    if ((e = cudaMemcpyAsync(u_d, u, sizeof(double) * ns * n, cudaMemcpyHostToDevice, c->stream))) return e;
    if ((e = launch_prior_transform(slots_d, ns, u_d, (int)n, th_d, c->stream, sky))) return e;
    if ((e = cudaMemcpyAsync(theta, th_d, sizeof(double) * SWIG_N_PARAMS * n, cudaMemcpyDeviceToHost, c->stream)))
      return e;
    return cudaStreamSynchronize(c->stream);
  };
  const cudaError_t e = run();
  if (slots_d) cudaFree(slots_d);
  if (u_d) cudaFree(u_d);
  if (th_d) cudaFree(th_d);
  if (e != cudaSuccess) return fail(c, SWIG_E_CUDA, std::string("prior transform: ") + cudaGetErrorString(e));
  ++c->n_launches;
  return SWIG_OK;
}

}  // extern "C"
