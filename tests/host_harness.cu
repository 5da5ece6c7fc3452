// Host-only harness over the library's preparation code, for the CPU tests:
// it compiles the C-ABI source into a small program that calls the pure host
// routines (no device call is made, so it runs without a GPU) and prints
// their results as JSON for comparison with numpy and the oracle.
//
//   host_harness edges F_MIN F_MAX DF N_BINS SPACING   heterodyne bin-edge indices
//   host_harness gl N                                  Gauss-Legendre nodes, weights
//   host_harness frame AX AY AZ BX BY BZ GMST          detector sky frame (b -> a)
//   host_harness tiles F_MIN F_MAX DF                  phase tiles of the mixed path
//   host_harness slices F_MIN F_MAX DF NDET SMS (LO HI)x6   slices of the persistent kernel over the
//                                                      tiles of a prior box (Mc q chi1 chi2 L1 L2)
//   host_harness coeffs MC Q CHI1 CHI2 LAM1 LAM2       TaylorF2 phase-basis coefficients
//                                                      (the host/device set-up code)
//   host_harness amp MC                                SPA amplitude at 1 Mpc
//   host_harness logi0 X...                            log I0(x) (FP64) and log(I0(x) e^-x) (FP32)
//   host_harness distmarg KIND LO HI PM ZRE ZIM H DD   distance-marginal logL (64-node rule)
//   host_harness prior KIND LO HI U...                 prior inverse CDF of one slot
//   host_harness sky AX AY AZ BX BY BZ GMST AZI ZEN    frame (azimuth, zenith) -> (RA, Dec)
//   host_harness priormap < SLOTS ROWS                 13 slots (kind mode lo hi value) then
//                                                      rows of sampled unit-cube coordinates
//   host_harness abi                                   sizes and field offsets of the C-ABI structs
//   host_harness nufft NT DT < NE FE...                 time-pass NUFFT tables for edge frequencies FE
//   host_harness tmtables < NB NDET DT EDGES A01       time-marginalisation edge tables
//   host_harness hetsum < N NB NDET DF F IDX (DATA PSD H0)xNDET   heterodyne summary data
//   host_harness weights F_MIN F_MAX DF NDET STRIDE < (DATA PSD)xNDET   full-grid data weights
//   host_harness hetchunks F_MIN F_MAX DF N_BINS SPACING   heterodyne chunk anchor tables
//   host_harness nufftpieces NT DT < NE FE...           gather pieces and stage-major FFT twiddles of
//                                                      the time-pass NUFFT
#include "../paper_2607_28265_gb300/csrc/capi.cu"

#include <cstddef>
#include <cstdlib>

#define SWIG_FIELD(T, f) std::printf("%s[\"%s\", %zu]", first ? "" : ", ", #f, offsetof(T, f)), first = false

static void print_array(const char* name, const double* v, int n, bool last) {
  std::printf("\"%s\": [", name);
  for (int i = 0; i < n; ++i) std::printf("%s%.17g", i ? ", " : "", v[i]);
  std::printf("]%s", last ? "" : ", ");
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const std::string what = argv[1];
  if (what == "edges" && argc == 7) {
    swig_ctx c;
    if (swig_set_grid(&c, std::atof(argv[2]), std::atof(argv[3]), std::atof(argv[4])) != SWIG_OK) return 3;
    std::vector<double> f((size_t)c.n_bins);
    for (int64_t k = 0; k < c.n_bins; ++k) f[(size_t)k] = (double)(c.k_min + k) * c.df;
    const std::vector<int> idx = het_edge_indices(f, std::atoi(argv[5]), std::atoi(argv[6]));
    std::printf("{\"k_min\": %lld, \"n_bins\": %lld, \"idx\": [", (long long)c.k_min, (long long)c.n_bins);
    for (size_t i = 0; i < idx.size(); ++i) std::printf("%s%d", i ? ", " : "", idx[i]);
    std::printf("]}\n");
    return 0;
  }
  if (what == "gl" && argc == 3) {
    const int n = std::atoi(argv[2]);
    std::vector<double> x(n), w(n);
    gauss_legendre(n, x.data(), w.data());
    std::printf("{");
    print_array("x", x.data(), n, false);
    print_array("w", w.data(), n, true);
    std::printf("}\n");
    return 0;
  }
  if (what == "frame" && argc == 9) {
    swig_ctx c;
    for (int k = 0; k < 3; ++k) {
      c.vertex[0][k] = std::atof(argv[2 + k]);
      c.vertex[1][k] = std::atof(argv[5 + k]);
    }
    c.det_set[0] = c.det_set[1] = true;
    c.sky_a = 0;
    c.sky_b = 1;
    c.gmst = std::atof(argv[8]);
    c.params[9] = swig_param{SWIG_PRIOR_UNIFORM, 0.0, 2.0 * kPi, SWIG_MODE_SAMPLE, 0.0, 4};
    c.params[10] = swig_param{SWIG_PRIOR_SINE, 0.0, kPi, SWIG_MODE_SAMPLE, 0.0, 4};
    SkyFrame F;
    if (make_sky_frame(&c, &F) != SWIG_OK) return 4;
    std::printf("{");
    print_array("ex", F.ex, 3, false);
    print_array("ey", F.ey, 3, false);
    print_array("ez", F.ez, 3, true);
    std::printf("}\n");
    return 0;
  }
  if (what == "coeffs" && argc == 8) {
    double cc[NBASIS];
    taylorf2_basis_coeffs(std::atof(argv[2]), std::atof(argv[3]), std::atof(argv[4]), std::atof(argv[5]),
                          std::atof(argv[6]), std::atof(argv[7]), cc);
    std::printf("{");
    print_array("c", cc, NBASIS, true);
    std::printf("}\n");
    return 0;
  }
  if (what == "amp" && argc == 3) {
    std::printf("{\"amp\": %.17g}\n", amplitude_per_mpc(std::atof(argv[2])));
    return 0;
  }
  if (what == "logi0" && argc >= 3) {
    std::vector<double> a, b;
    for (int i = 2; i < argc; ++i) {
      const double x = std::atof(argv[i]);
      a.push_back(log_bessel_i0(x));
      b.push_back((double)log_i0e_f32((float)x));
    }
    std::printf("{");
    print_array("log_i0", a.data(), (int)a.size(), false);
    print_array("log_i0e_f32", b.data(), (int)b.size(), true);
    std::printf("}\n");
    return 0;
  }
  if (what == "distmarg" && argc == 10) {
    LikeConst L{};
    L.dist_marg = 1;
    L.d_kind = std::atoi(argv[2]);
    L.d_lo = std::atof(argv[3]);
    L.d_hi = std::atof(argv[4]);
    L.phase_marg = std::atoi(argv[5]);
    L.DD = std::atof(argv[9]);
    gauss_legendre(kGaussLegendre, L.gl_x, L.gl_w);
    std::printf("{\"logl\": %.17g}\n", distance_marg_logl(L, std::atof(argv[6]), std::atof(argv[7]), std::atof(argv[8])));
    return 0;
  }
  if (what == "prior" && argc >= 6) {
    const PriorSlot s = make_prior_slot(std::atoi(argv[2]), SWIG_MODE_SAMPLE, std::atof(argv[3]), std::atof(argv[4]), 0.0);
    std::vector<double> x;
    for (int i = 5; i < argc; ++i) x.push_back(prior_slot_inverse(s, std::atof(argv[i])));
    std::printf("{");
    print_array("x", x.data(), (int)x.size(), true);
    std::printf("}\n");
    return 0;
  }
  if (what == "sky" && argc == 11) {
    swig_ctx c;
    for (int k = 0; k < 3; ++k) {
      c.vertex[0][k] = std::atof(argv[2 + k]);
      c.vertex[1][k] = std::atof(argv[5 + k]);
    }
    c.det_set[0] = c.det_set[1] = true;
    c.sky_a = 0;
    c.sky_b = 1;
    c.gmst = std::atof(argv[8]);
    c.params[9] = swig_param{SWIG_PRIOR_UNIFORM, 0.0, 2.0 * kPi, SWIG_MODE_SAMPLE, 0.0, 4};
    c.params[10] = swig_param{SWIG_PRIOR_SINE, 0.0, kPi, SWIG_MODE_SAMPLE, 0.0, 4};
    SkyFrame F;
    if (make_sky_frame(&c, &F) != SWIG_OK) return 4;
    double ra, dec;
    sky_frame_to_radec(F, std::atof(argv[9]), std::atof(argv[10]), &ra, &dec);
    std::printf("{\"ra\": %.17g, \"dec\": %.17g}\n", ra, dec);
    return 0;
  }
  if (what == "priormap" && argc == 2) {
    PriorSlot slots[SWIG_N_PARAMS];
    int n_sampled = 0;
    for (int i = 0; i < SWIG_N_PARAMS; ++i) {
      int kind, mode;
      double lo, hi, value;
      if (std::scanf("%d %d %lf %lf %lf", &kind, &mode, &lo, &hi, &value) != 5) return 5;
      slots[i] = make_prior_slot(kind, mode, lo, hi, value);
      n_sampled += mode == SWIG_MODE_SAMPLE;
    }
    std::printf("{\"theta\": [");
    for (int row = 0;; ++row) {
      double u[SWIG_N_PARAMS];
      int got = 0;
      for (int j = 0; j < n_sampled; ++j) got += std::scanf("%lf", &u[j]);
      if (got != n_sampled) break;
      double th[SWIG_N_PARAMS];
      prior_map(slots, u, th);
      std::printf("%s[", row ? ", " : "");
      for (int j = 0; j < SWIG_N_PARAMS; ++j) std::printf("%s%.17g", j ? ", " : "", th[j]);
      std::printf("]");
    }
    std::printf("]}\n");
    return 0;
  }
  if (what == "weights" && argc == 7) {
    swig_ctx c;
    if (swig_set_grid(&c, std::atof(argv[2]), std::atof(argv[3]), std::atof(argv[4])) != SWIG_OK) return 3;
    const int n_det = std::atoi(argv[5]), stride = std::atoi(argv[6]);
    const int64_t n = c.n_bins;
    for (int i = 0; i < n_det; ++i) {
      std::vector<double> d(2 * (size_t)n), s((size_t)n);
      for (double& v : d)
        if (std::scanf("%lf", &v) != 1) return 5;
      for (double& v : s)
        if (std::scanf("%lf", &v) != 1) return 5;
      if (swig_set_data(&c, i, d.data(), n) != SWIG_OK || swig_set_psd(&c, i, s.data(), n) != SWIG_OK) return 6;
    }
    std::vector<double> dre, dim, sre, sim;
    double K[SWIG_MAX_DET], dmax[SWIG_MAX_DET], dd;
    weight_data(&c, n_det, dre, dim, K, &dd, dmax);
    for (size_t k = 0; k < dre.size(); k += (size_t)stride) {
      sre.push_back(dre[k]);
      sim.push_back(dim[k]);
    }
    std::printf("{\"dd\": %.17g, ", dd);
    print_array("K", K, n_det, false);
    print_array("dmax", dmax, n_det, false);
    print_array("dre", sre.data(), (int)sre.size(), false);
    print_array("dim", sim.data(), (int)sim.size(), true);
    std::printf("}\n");
    return 0;
  }
  if (what == "hetsum" && argc == 2) {
    int n, nb, n_det;
    double df;
    if (std::scanf("%d %d %d %lf", &n, &nb, &n_det, &df) != 4 || n_det < 1 || n_det > SWIG_MAX_DET) return 5;
    std::vector<double> f(n);
    std::vector<int> idx(nb + 1);
    for (double& v : f)
      if (std::scanf("%lf", &v) != 1) return 5;
    for (int& v : idx)
      if (std::scanf("%d", &v) != 1) return 5;
    std::vector<double> data[SWIG_MAX_DET], psd[SWIG_MAX_DET];
    std::vector<double2> h0((size_t)n_det * n);
    for (int i = 0; i < n_det; ++i) {
      data[i].resize(2 * (size_t)n);
      psd[i].resize(n);
      for (double& v : data[i])
        if (std::scanf("%lf", &v) != 1) return 5;
      for (double& v : psd[i])
        if (std::scanf("%lf", &v) != 1) return 5;
      for (int k = 0; k < n; ++k)
        if (std::scanf("%lf %lf", &h0[(size_t)i * n + k].x, &h0[(size_t)i * n + k].y) != 2) return 5;
    }
    std::vector<float4> coef;
    std::vector<float2> coefB;
    std::vector<double> a01;
    het_summary(f, idx, nb, n_det, df, data, psd, h0, coef, coefB, a01);
    std::printf("{");
    print_array("a01", a01.data(), (int)a01.size(), false);
    std::vector<double> bb;
    for (const float2& v : coefB) {
      bb.push_back(v.x);
      bb.push_back(v.y);
    }
    print_array("b01", bb.data(), (int)bb.size(), true);
    std::printf("}\n");
    return 0;
  }
  if (what == "tmtables" && argc == 2) {
    int nb, n_det;
    double dt;
    if (std::scanf("%d %d %lf", &nb, &n_det, &dt) != 3) return 5;
    std::vector<double> f(nb + 1), a01((size_t)n_det * nb * 4);
    std::vector<int> idx(nb + 1);
    for (int q = 0; q <= nb; ++q) {
      if (std::scanf("%lf", &f[q]) != 1) return 5;
      idx[q] = q;
    }
    for (double& v : a01)
      if (std::scanf("%lf", &v) != 1) return 5;
    std::vector<float2> g, w;
    het_tm_tables(a01, f, idx, nb, n_det, dt, g, w);
    std::printf("{\"g\": [");
    for (size_t k = 0; k < g.size(); ++k) std::printf("%s%.9g, %.9g", k ? ", " : "", g[k].x, g[k].y);
    std::printf("], \"w\": [");
    for (size_t k = 0; k < w.size(); ++k) std::printf("%s%.9g, %.9g", k ? ", " : "", w[k].x, w[k].y);
    std::printf("]}\n");
    return 0;
  }
  if (what == "abi" && argc == 2) {
    bool first = true;
    std::printf("{\"swig_param\": {\"size\": %zu, \"fields\": [", sizeof(swig_param));
    SWIG_FIELD(swig_param, kind); SWIG_FIELD(swig_param, lo); SWIG_FIELD(swig_param, hi);
    SWIG_FIELD(swig_param, mode); SWIG_FIELD(swig_param, value); SWIG_FIELD(swig_param, block);
    first = true;
    std::printf("]}, \"swig_sampler_cfg\": {\"size\": %zu, \"fields\": [", sizeof(swig_sampler_cfg));
    SWIG_FIELD(swig_sampler_cfg, nlive); SWIG_FIELD(swig_sampler_cfg, nrep); SWIG_FIELD(swig_sampler_cfg, sweeps);
    SWIG_FIELD(swig_sampler_cfg, steps_per_dim); SWIG_FIELD(swig_sampler_cfg, seed);
    SWIG_FIELD(swig_sampler_cfg, likelihood); SWIG_FIELD(swig_sampler_cfg, precision);
    SWIG_FIELD(swig_sampler_cfg, proposal); SWIG_FIELD(swig_sampler_cfg, het_bins);
    SWIG_FIELD(swig_sampler_cfg, het_spacing); SWIG_FIELD(swig_sampler_cfg, dlogz);
    SWIG_FIELD(swig_sampler_cfg, max_iter); SWIG_FIELD(swig_sampler_cfg, het_fiducial);
    SWIG_FIELD(swig_sampler_cfg, learn_mix); SWIG_FIELD(swig_sampler_cfg, learn_lr);
    SWIG_FIELD(swig_sampler_cfg, learn_steps); SWIG_FIELD(swig_sampler_cfg, learn_interval);
    SWIG_FIELD(swig_sampler_cfg, tmarg_nodes); SWIG_FIELD(swig_sampler_cfg, cache_off);
    SWIG_FIELD(swig_sampler_cfg, flow_parts); SWIG_FIELD(swig_sampler_cfg, stepout_one_end);
    first = true;
    std::printf("]}, \"swig_result\": {\"size\": %zu, \"fields\": [", sizeof(swig_result));
    SWIG_FIELD(swig_result, logz); SWIG_FIELD(swig_result, logz_err); SWIG_FIELD(swig_result, info);
    SWIG_FIELD(swig_result, ess); SWIG_FIELD(swig_result, wall_s); SWIG_FIELD(swig_result, n_dead);
    SWIG_FIELD(swig_result, n_iter); SWIG_FIELD(swig_result, n_evals); SWIG_FIELD(swig_result, n_sweep_evals);
    SWIG_FIELD(swig_result, status);
    std::printf("]}}\n");
    return 0;
  }
  if (what == "nufft" && argc == 4) {
    int ne = 0;
    if (std::scanf("%d", &ne) != 1 || ne < 1) return 3;
    std::vector<double> fe(ne);
    for (int e = 0; e < ne; ++e)
      if (std::scanf("%lf", &fe[e]) != 1) return 3;
    int M = 0, j0 = 0;
    std::vector<int> ptr, edge;
    std::vector<float> wt, corr;
    std::vector<float2> tw;
    het_nufft_tables(fe, std::atoi(argv[2]), std::atof(argv[3]), kNufftWidth, &M, &j0, ptr, edge, wt, corr, tw);
    std::printf("{\"M\": %d, \"j0\": %d, \"ptr\": [", M, j0);
    for (size_t q = 0; q < ptr.size(); ++q) std::printf("%s%d", q ? ", " : "", ptr[q]);
    std::printf("], \"edge\": [");
    for (size_t q = 0; q < edge.size(); ++q) std::printf("%s%d", q ? ", " : "", edge[q]);
    std::printf("], \"wt\": [");
    for (size_t q = 0; q < wt.size(); ++q) std::printf("%s%.9g", q ? ", " : "", wt[q]);
    std::printf("], \"corr\": [");
    for (size_t q = 0; q < corr.size(); ++q) std::printf("%s%.9g", q ? ", " : "", corr[q]);
    std::printf("]}\n");
    return 0;
  }
  if (what == "hetchunks" && argc == 7) {
    swig_ctx c;
    if (swig_set_grid(&c, std::atof(argv[2]), std::atof(argv[3]), std::atof(argv[4])) != SWIG_OK) return 3;
    std::vector<double> f((size_t)c.n_bins);
    for (int64_t k = 0; k < c.n_bins; ++k) f[(size_t)k] = (double)(c.k_min + k) * c.df;
    const std::vector<int> idx = het_edge_indices(f, std::atoi(argv[5]), std::atoi(argv[6]));
    const int nb = (int)idx.size() - 1;
    std::vector<float> ct, dfe;
    const int nc = het_chunk_tables(f, idx, nb, ct, dfe);
    std::printf("{\"nb\": %d, \"nc\": %d, \"rows\": %d, \"nbasis\": %d, \"poly\": %d, \"row\": {\"val_hi\": %d, "
                "\"val_lo\": %d, \"d1_hi\": %d, \"d1_lo\": %d, \"poly\": %d, \"fa_hi\": %d, \"fa_lo\": %d, \"inv_s\": %d, "
                "\"bnd\": %d}, \"fe\": [",
                nb, nc, (int)HC_ROWS, (int)NBASIS, kHetPoly, (int)HC_VAL_HI, (int)HC_VAL_LO, (int)HC_D1_HI,
                (int)HC_D1_LO, (int)HC_POLY, (int)HC_FA_HI, (int)HC_FA_LO, (int)HC_INV_S, (int)HC_BND);
    for (int e = 0; e <= nb; ++e) std::printf("%s%.17g", e ? ", " : "", f[idx[e]]);
    std::printf("], \"ct\": [");
    for (size_t q = 0; q < ct.size(); ++q) std::printf("%s%.9g", q ? ", " : "", ct[q]);
    std::printf("], \"dfe\": [");
    for (size_t q = 0; q < dfe.size(); ++q) std::printf("%s%.9g", q ? ", " : "", dfe[q]);
    std::printf("]}\n");
    return 0;
  }
  if (what == "nufftpieces" && argc == 4) {
    int ne = 0;
    if (std::scanf("%d", &ne) != 1 || ne < 1) return 3;
    std::vector<double> fe(ne);
    for (int e = 0; e < ne; ++e)
      if (std::scanf("%lf", &fe[e]) != 1) return 3;
    int M = 0, j0 = 0;
    std::vector<int> ptr, edge;
    std::vector<float> wt, corr;
    std::vector<float2> tw;
    het_nufft_tables(fe, std::atoi(argv[2]), std::atof(argv[3]), kNufftWidth, &M, &j0, ptr, edge, wt, corr, tw);
    std::vector<int4> piece, point;
    if (!ptr.empty()) nufft_pieces(ptr, edge, M, piece, point);
    const std::vector<float2> tws = nufft_stage_twiddles(tw, M);
    std::printf("{\"M\": %d, \"max_piece\": %d, \"tw\": [", M, kNufftPiece);
    for (size_t q = 0; q < tws.size(); ++q) std::printf("%s[%.9g, %.9g]", q ? ", " : "", tws[q].x, tws[q].y);
    std::printf("], \"ptr\": [");
    for (size_t q = 0; q < ptr.size(); ++q) std::printf("%s%d", q ? ", " : "", ptr[q]);
    std::printf("], \"edge\": [");
    for (size_t q = 0; q < edge.size(); ++q) std::printf("%s%d", q ? ", " : "", edge[q]);
    std::printf("], \"piece\": [");
    for (size_t q = 0; q < piece.size(); ++q)
      std::printf("%s[%d, %d, %d]", q ? ", " : "", piece[q].x, piece[q].y, piece[q].z);
    std::printf("], \"point\": [");
    for (size_t q = 0; q < point.size(); ++q)
      std::printf("%s[%d, %d, %d]", q ? ", " : "", point[q].x, point[q].y, point[q].z);
    std::printf("]}\n");
    return 0;
  }
  if (what == "slices" && argc == 19) {
    swig_ctx c;
    if (swig_set_grid(&c, std::atof(argv[2]), std::atof(argv[3]), std::atof(argv[4])) != SWIG_OK) return 3;
    for (int i = 0; i < 6; ++i) {
      c.params[i].mode = SWIG_MODE_SAMPLE;
      c.params[i].lo = std::atof(argv[7 + 2 * i]);
      c.params[i].hi = std::atof(argv[8 + 2 * i]);
    }
    c.prior_set = true;
    std::vector<TileInfo> tiles;
    std::vector<TileBasis> basis;
    plan_tiles(&c, tiles, basis);
    std::vector<int> sb;
    int max_bins = 0;
    plan_slices(c.n_bins, std::atoi(argv[5]), std::atoi(argv[6]), tiles, sb, &max_bins);
    std::printf("{\"max_bins\": %d, \"slice_begin\": [", max_bins);
    for (size_t q = 0; q < sb.size(); ++q) std::printf("%s%d", q ? ", " : "", sb[q]);
    std::printf("], \"tiles\": [");
    for (size_t t = 0; t < tiles.size(); ++t) std::printf("%s[%d, %d]", t ? ", " : "", tiles[t].k0, tiles[t].nbins);
    std::printf("]}\n");
    return 0;
  }
  if (what == "tiles" && argc == 5) {
    swig_ctx c;
    if (swig_set_grid(&c, std::atof(argv[2]), std::atof(argv[3]), std::atof(argv[4])) != SWIG_OK) return 3;
    double cmax[NBASIS];
    coefficient_bounds(&c, cmax);
    std::vector<TileInfo> tiles;
    std::vector<TileBasis> basis;
    plan_tiles(&c, tiles, basis);
    std::printf("{\"k_min\": %lld, ", (long long)c.k_min);
    print_array("cmax", cmax, NBASIS, false);
    std::printf("\"tiles\": [");
    for (size_t t = 0; t < tiles.size(); ++t) {
      const TileInfo& ti = tiles[t];
      const TileBasis& tb = basis[t];
      std::printf("%s{\"k0\": %d, \"nbins\": %d, \"inv_T\": %.9g, ", t ? ", " : "", ti.k0, ti.nbins, ti.inv_T);
      double v[NBASIS], s[NBASIS];
      for (int j = 0; j < NBASIS; ++j) {
        v[j] = (double)tb.val_hi[j] + (double)tb.val_lo[j];
        s[j] = (double)tb.slope_hi[j] + (double)tb.slope_lo[j];
      }
      print_array("val", v, NBASIS, false);
      print_array("slope", s, NBASIS, false);
      std::printf("\"poly\": [");
      for (int m = 0; m < kNumPoly; ++m) {
        double pm[NBASIS];
        for (int j = 0; j < NBASIS; ++j) pm[j] = tb.poly[m][j];
        std::printf("%s[", m ? ", " : "");
        for (int j = 0; j < NBASIS; ++j) std::printf("%s%.9g", j ? ", " : "", pm[j]);
        std::printf("]");
      }
      std::printf("]}");
    }
    std::printf("]}\n");
    return 0;
  }
  return 2;
}
