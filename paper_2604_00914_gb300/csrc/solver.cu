// AdaPolySI on one GPU: set-up (Sec. 3.4 bounds, Sec. 2.2 coefficients,
// Eq. (compute_k_1)), then per outer iteration (Alg. 4): filter by Clenshaw
// (Alg. 2) in FP64 or FP32, orthogonalisation against the locked vectors and
// CholQR2, Rayleigh-Ritz, residuals, the spurious test (Eq. (tau_s)), locking
// and the next degree (Alg. 3).  The dense and sparse work runs in the
// library's kernels; the host handles the p Ritz values and index sets of each
// iteration (one device-to-host transfer of 2 p doubles per iteration).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <numeric>

#include "solver_impl.cuh"

namespace apf {

// ---- Sec. 3.4: spectrum bounds ----------------------------------------------------
template <class T>
static void spectrum_bounds_t(apf_ctx* ctx, const apf_matrix* A, int steps, uint64_t seed,
                              double pad, double out[6]) {
  const int64_t n = A->n;
  const int m = (int)std::min<int64_t>(steps, n);
  APF_REQUIRE(m >= 1, APF_ERR_ARG);
  const T* vals = static_cast<const T*>(A->vals);
  DBuf Q((size_t)n * (m + 1) * sizeof(T), ctx->stream, true);
  DBuf w((size_t)n * sizeof(T), ctx->stream, true);
  DBuf cf((size_t)(m + 1) * sizeof(T), ctx->stream, true);
  DBuf ab((size_t)(2 * m + 2) * sizeof(double), ctx->stream, true);
  T* q = Q.as<T>();
  double* alpha = ab.as<double>();
  double* beta = alpha + m + 1;
  random_block<T>(ctx, seed, 2u, n, 1, q, 1);
  norm2<T>(ctx, n, q, beta + m);
  scale_vec_by_inv<T>(ctx, n, q, beta + m, q);
  std::vector<double> ha, hb;
  for (int j = 0; j < m; ++j) {
    spmv<T>(ctx, n, A->rowptr, A->colidx, vals, q + (int64_t)j * n, w.as<T>());
    lanczos_update<T>(ctx, n, j, q, w.as<T>(), alpha, beta);
    for (int pass = 0; pass < 2; ++pass) {
      dot_many<T>(ctx, n, j + 1, q, w.as<T>(), cf.as<T>());
      axpy_many<T>(ctx, n, j + 1, q, cf.as<T>(), w.as<T>());
    }
    norm2<T>(ctx, n, w.as<T>(), beta + j);
    double hab[2];
    APF_CUDA(cudaMemcpyAsync(&hab[0], alpha + j, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    APF_CUDA(cudaMemcpyAsync(&hab[1], beta + j, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    APF_CUDA(cudaStreamSynchronize(ctx->stream));
    ha.push_back(hab[0]);
    hb.push_back(hab[1]);
    double amax = 1.0;
    for (double v : ha) amax = std::max(amax, fabs(v));
    if (j == m - 1 || hab[1] <= 1e-14 * amax) break;
    scale_vec_by_inv<T>(ctx, n, w.as<T>(), beta + j, q + (int64_t)(j + 1) * n);
  }
  const int mm = (int)ha.size();
  // tridiagonal T_m, eigenvalues and last components of its eigenvectors
  std::vector<double> Th((size_t)mm * mm, 0.0);
  for (int i = 0; i < mm; ++i) {
    Th[(size_t)i * mm + i] = ha[(size_t)i];
    if (i + 1 < mm) Th[(size_t)i * mm + i + 1] = Th[(size_t)(i + 1) * mm + i] = hb[(size_t)i];
  }
  DBuf Td((size_t)mm * mm * sizeof(double), ctx->stream, false);
  DBuf Ud((size_t)mm * mm * sizeof(double), ctx->stream, false);
  DBuf wd((size_t)mm * sizeof(double), ctx->stream, false);
  APF_CUDA(cudaMemcpyAsync(Td.p, Th.data(), Th.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  eigh_jacobi<double>(ctx, mm, Td.as<double>(), mm, wd.as<double>(), Ud.as<double>(), mm);
  std::vector<double> hw((size_t)mm), hU((size_t)mm * mm);
  APF_CUDA(cudaMemcpyAsync(hw.data(), wd.p, hw.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  APF_CUDA(cudaMemcpyAsync(hU.data(), Ud.p, hU.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  const int derr = fetch_device_error(ctx);
  if (derr == DEV_EIGH_NOCONV) throw ApfError{APF_ERR_EIGH, "Lanczos tridiagonal eigensolver"};
  if (derr == DEV_BARRIER_TIMEOUT) throw ApfError{APF_ERR_TIMEOUT, "eigensolver barrier"};
  const double th_lo = hw[0], th_hi = hw[(size_t)mm - 1];
  const double blast = hb[(size_t)mm - 1];
  const double res_lo = fabs(blast * hU[(size_t)(mm - 1) * mm + 0]);
  const double res_hi = fabs(blast * hU[(size_t)(mm - 1) * mm + (mm - 1)]);
  const double spread = th_hi - th_lo;
  double lmax = th_hi + res_hi + pad * spread;
  double lmin = th_lo - res_lo - pad * spread;
  lmax = std::min(lmax, A->gersh_hi);
  lmin = std::max(lmin, A->gersh_lo);
  out[0] = lmin;
  out[1] = lmax;
  out[2] = th_lo;
  out[3] = th_hi;
  out[4] = A->gersh_lo;
  out[5] = A->gersh_hi;
}

void spectrum_bounds(apf_ctx* ctx, const apf_matrix* A, int steps, uint64_t seed, double pad,
                     double out[6]) {
  if (A->dtype == APF_C128) spectrum_bounds_t<double2>(ctx, A, steps, seed, pad, out);
  else spectrum_bounds_t<double>(ctx, A, steps, seed, pad, out);
}


template <class T>
static void solve_t(apf_ctx* ctx, const apf_matrix* A, const apf_params* prm, apf_result* out) {
  using clock = std::chrono::steady_clock;
  const auto t_start = clock::now();
  const int64_t n = A->n;
  APF_REQUIRE(prm->p >= 0 && prm->p <= n && prm->p <= APF_MAX_P, APF_ERR_ARG);
  APF_REQUIRE(prm->p > 0 || (prm->init_block == nullptr && prm->mu > 0.0 && prm->trace_probes >= 1), APF_ERR_ARG);
  APF_REQUIRE(prm->a < prm->b, APF_ERR_ARG);
  APF_REQUIRE(prm->max_iter >= 1, APF_ERR_ARG);
  APF_REQUIRE(prm->filter_precision >= APF_FILTER_F64 && prm->filter_precision <= APF_FILTER_F32_DEFECT,
              APF_ERR_ARG);
  const int64_t launches0 = ctx->launches;
  apf_stats st{};

  // set-up (Alg. 4): bounds, map, degrees, coefficients, initial block
  const Bounds bd = setup_bounds(ctx, A, prm);
  IntervalState<T> S;
  S.setup_filter(prm, prm->a, prm->b, bd.l1, bd.l2);
  int64_t p = prm->p;
  if (p == 0) {  // Sec. 3.4: p = ceil(mu e~) from the estimated count
    st.trace_estimate = count_estimates<T>(ctx, A, prm->filter_precision, bd.l1, bd.l2, {&S.coef},
                                           prm->trace_probes, prm->seed)[0];
    p = subspace_size(st.trace_estimate, prm->mu, n);
  }
  st.p_used = p;
  SmallWork<T> sw;
  sw.init(p, ctx->stream);
  S.init_block(ctx, A, prm, p, 1u, sw);
  st.k1 = S.k1;
  st.k_max = S.kmax;
  st.lambda_min = bd.lmin;
  st.lambda_max = bd.lmax;
  st.norm_a = bd.normA;
  FilterState<T> fs;
  fs.init(ctx, A, S.ld, bd.l1, bd.l2, S.coef, prm->filter_precision);
  fs.graphs_on = prm->filter_graphs != 0;
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  st.ms_setup = std::chrono::duration<double, std::milli>(clock::now() - t_start).count();

  EventPool evp;
  std::vector<IterEv> iev;
  std::vector<double> hist;
  apf_status status = APF_ERR_NO_CONVERGENCE;
  FilterCount fc;
  double deg_sum = 0.0;
  int iters = 0;
  for (int it = 1; it <= prm->max_iter; ++it) {
    IterEv ev{evp.get(), evp.get(), evp.get(), evp.get(), evp.get(), evp.get()};
    iev.push_back(ev);
    APF_CUDA(cudaEventRecord(ev.e0, ctx->stream));
    // filtering (Alg. 2)
    const bool defect = S.have_ritz && prm->filter_precision == APF_FILTER_F32_DEFECT;
    fs.apply(S.ki, S.Vh.template as<T>(), defect ? S.AVh.template as<T>() : nullptr, defect ? S.w : nullptr,
             S.pa, S.X.template as<T>(), ev.f0, ev.f1, &fc);
    st.spmv_columns += (int64_t)S.ki * S.pa + 2 * S.pa;
    deg_sum += S.ki;
    ++iters;
    APF_CUDA(cudaEventRecord(ev.e1, ctx->stream));
    // orthogonalisation, Rayleigh-Ritz, residuals
    S.orth(ctx, A, sw, prm->gram_tensor_cores != 0);
    APF_CUDA(cudaEventRecord(ev.e2, ctx->stream));
    check_device_after_rr(ctx);
    S.check(ctx, A, prm, bd.l1, bd.l2, bd.normA);
    APF_CUDA(cudaEventRecord(ev.e3, ctx->stream));
    hist.insert(hist.end(), S.rec.begin(), S.rec.end());
    if (S.done) {
      status = APF_OK;
      break;
    }
    if (S.pa == 0) break;
  }
  finish_stats(ctx, iev, fc, iters, deg_sum, &st);
  assemble_result<T>(ctx, A, {&S}, bd.normA, out);
  st.max_residual = 0.0;
  for (double r : out->res) st.max_residual = std::max(st.max_residual, r);
  st.gpu_launches = ctx->launches - launches0;
  st.ms_total = std::chrono::duration<double, std::milli>(clock::now() - t_start).count();
  out->history = hist;
  out->stats = st;
  if (status != APF_OK) throw ApfError{status, "no convergence"};
}

// Spectrum slicing: disjoint intervals [a_s, b_s] with their own subspaces
// and filters (Sec. 1: the slices are independent problems).  One filter
// application serves all slices: their blocks are concatenated with the
// higher degrees first, every column carries its slice's coefficients, and a
// slice of degree k_s joins the recurrence at step k_s, so all slices finish
// on the same step.  Orthogonalisation, Rayleigh-Ritz, the spurious rule and
// locking run per slice, exactly as in a single solve.
template <class T>
static void solve_slices_t(apf_ctx* ctx, const apf_matrix* A, int ns, const double* a, const double* b,
                           const int64_t* p, const apf_params* prm, apf_result* out) {
  using clock = std::chrono::steady_clock;
  const auto t_start = clock::now();
  const int64_t n = A->n;
  APF_REQUIRE(ns >= 1 && a && b && p, APF_ERR_ARG);
  APF_REQUIRE(prm->max_iter >= 1 && prm->init_block == nullptr, APF_ERR_ARG);
  APF_REQUIRE(prm->filter_precision >= APF_FILTER_F64 && prm->filter_precision <= APF_FILTER_F32_DEFECT,
              APF_ERR_ARG);
  bool any_estimate = false;
  for (int s = 0; s < ns; ++s) {
    APF_REQUIRE(p[s] >= 0 && a[s] < b[s], APF_ERR_ARG);
    any_estimate = any_estimate || p[s] == 0;
  }
  APF_REQUIRE(!any_estimate || (prm->mu > 0.0 && prm->trace_probes >= 1), APF_ERR_ARG);
  // slices in ascending order must not overlap
  std::vector<int> by_a((size_t)ns);
  std::iota(by_a.begin(), by_a.end(), 0);
  std::stable_sort(by_a.begin(), by_a.end(), [&](int u, int v) { return a[u] < a[v]; });
  for (int i = 1; i < ns; ++i) APF_REQUIRE(b[by_a[(size_t)i - 1]] < a[by_a[(size_t)i]], APF_ERR_ARG);
  const int64_t launches0 = ctx->launches;
  apf_stats st{};

  const Bounds bd = setup_bounds(ctx, A, prm);
  std::vector<IntervalState<T>> S((size_t)ns);
  for (int s = 0; s < ns; ++s) S[(size_t)s].setup_filter(prm, a[s], b[s], bd.l1, bd.l2);
  // Sec. 3.4 for the slices without a size: their counts in one batched filter pass
  std::vector<int64_t> ps(p, p + ns);
  if (any_estimate) {
    std::vector<const std::vector<double>*> cs;
    std::vector<int> which;
    for (int s = 0; s < ns; ++s)
      if (p[s] == 0) { cs.push_back(&S[(size_t)s].coef); which.push_back(s); }
    const std::vector<double> e = count_estimates<T>(ctx, A, prm->filter_precision, bd.l1, bd.l2, cs,
                                                     prm->trace_probes, prm->seed);
    for (size_t i = 0; i < which.size(); ++i) {
      ps[(size_t)which[i]] = subspace_size(e[i], prm->mu, n);
      st.trace_estimate += e[i];
    }
  }
  int64_t ptot = 0, pmax = 0;
  for (int s = 0; s < ns; ++s) {
    ptot += ps[(size_t)s];
    pmax = std::max(pmax, ps[(size_t)s]);
  }
  APF_REQUIRE(ptot <= n && ptot <= APF_MAX_SUM_P, APF_ERR_ARG);
  st.p_used = ptot;
  SmallWork<T> sw;
  sw.init(pmax, ctx->stream);
  std::vector<double> coef_all;
  std::vector<int64_t> coff((size_t)ns);
  for (int s = 0; s < ns; ++s) {
    S[(size_t)s].init_block(ctx, A, prm, ps[(size_t)s], 1u + (uint32_t)s, sw);
    coff[(size_t)s] = (int64_t)coef_all.size();
    coef_all.insert(coef_all.end(), S[(size_t)s].coef.begin(), S[(size_t)s].coef.end());
    st.k1 = std::max(st.k1, S[(size_t)s].k1);
    st.k_max = std::max(st.k_max, S[(size_t)s].kmax);
  }
  st.lambda_min = bd.lmin;
  st.lambda_max = bd.lmax;
  st.norm_a = bd.normA;
  DBuf coef_dev(coef_all.size() * sizeof(double), ctx->stream, false);
  APF_CUDA(cudaMemcpyAsync(coef_dev.p, coef_all.data(), coef_all.size() * sizeof(double), cudaMemcpyHostToDevice,
                           ctx->stream));
  // the concatenated blocks
  const int64_t ldc = block_ld(ptot);
  const size_t blkc = (size_t)n * ldc * sizeof(T);
  DBuf Vc(blkc, ctx->stream, true), AVc(blkc, ctx->stream, true), Xc(blkc, ctx->stream, true);
  DBuf wc(sizeof(double) * (size_t)(ldc + 8), ctx->stream, true);
  FilterState<T> fs;
  fs.init(ctx, A, ldc, bd.l1, bd.l2, std::vector<double>(), prm->filter_precision);
  fs.graphs_on = prm->filter_graphs != 0;  // recurring applications of all slices replay as one graph
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  st.ms_setup = std::chrono::duration<double, std::milli>(clock::now() - t_start).count();

  EventPool evp;
  std::vector<IterEv> iev;
  std::vector<double> hist;
  FilterCount fc;
  double deg_sum = 0.0;
  int iters = 0;
  for (int it = 1; it <= prm->max_iter; ++it) {
    // active slices, highest degree first
    std::vector<int> act;
    for (int s = 0; s < ns; ++s)
      if (!S[(size_t)s].done && S[(size_t)s].pa > 0) act.push_back(s);
    if (act.empty()) break;
    std::stable_sort(act.begin(), act.end(), [&](int u, int v) { return S[(size_t)u].ki > S[(size_t)v].ki; });
    IterEv ev{evp.get(), evp.get(), evp.get(), evp.get(), evp.get(), evp.get()};
    iev.push_back(ev);
    APF_CUDA(cudaEventRecord(ev.e0, ctx->stream));
    // every active slice has Ritz values or none has (they start together)
    const bool defect = S[(size_t)act[0]].have_ritz && prm->filter_precision == APF_FILTER_F32_DEFECT;
    std::vector<int32_t> kc;
    std::vector<int64_t> co, off;
    int64_t pc = 0;
    for (int s : act) {
      IntervalState<T>& I = S[(size_t)s];
      off.push_back(pc);
      copy_block<T>(ctx, n, I.pa, I.Vh.template as<T>(), I.ld, Vc.as<T>() + pc, ldc);
      if (defect) {
        copy_block<T>(ctx, n, I.pa, I.AVh.template as<T>(), I.ld, AVc.as<T>() + pc, ldc);
        APF_CUDA(cudaMemcpyAsync(wc.as<double>() + pc, I.w, (size_t)I.pa * sizeof(double), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
      }
      for (int64_t c = 0; c < I.pa; ++c) {
        kc.push_back(I.ki);
        co.push_back(coff[(size_t)s]);
      }
      st.spmv_columns += (int64_t)I.ki * I.pa + 2 * I.pa;
      pc += I.pa;
    }
    if (pc < ldc) {  // padding columns of the concatenated blocks stay zero
      APF_CUDA(cudaMemset2DAsync(Vc.as<T>() + pc, ldc * sizeof(T), 0, (size_t)(ldc - pc) * sizeof(T), n, ctx->stream));
      if (defect)
        APF_CUDA(cudaMemset2DAsync(AVc.as<T>() + pc, ldc * sizeof(T), 0, (size_t)(ldc - pc) * sizeof(T), n,
                                   ctx->stream));
    }
    fs.apply_cols(kc, co, coef_dev.as<double>(), Vc.as<T>(), defect ? AVc.as<T>() : nullptr,
                  defect ? wc.as<double>() : nullptr, pc, Xc.as<T>(), ev.f0, ev.f1, &fc);
    for (size_t i = 0; i < act.size(); ++i) {
      IntervalState<T>& I = S[(size_t)act[i]];
      copy_block<T>(ctx, n, I.pa, Xc.as<T>() + off[i], ldc, I.X.template as<T>(), I.ld);
    }
    deg_sum += kc[0];
    ++iters;
    APF_CUDA(cudaEventRecord(ev.e1, ctx->stream));
    for (int s : act) S[(size_t)s].orth(ctx, A, sw, prm->gram_tensor_cores != 0);
    APF_CUDA(cudaEventRecord(ev.e2, ctx->stream));
    check_device_after_rr(ctx);
    std::vector<double> row = {(double)kc[0], 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int s : act) {
      IntervalState<T>& I = S[(size_t)s];
      I.check(ctx, A, prm, bd.l1, bd.l2, bd.normA);
      row[1] += I.rec[1];
      row[2] += I.rec[2];
      row[3] += I.rec[3];
      row[4] += I.rec[4];
      row[5] = std::max(row[5], I.rec[5]);
    }
    APF_CUDA(cudaEventRecord(ev.e3, ctx->stream));
    hist.insert(hist.end(), row.begin(), row.end());
  }
  finish_stats(ctx, iev, fc, iters, deg_sum, &st);
  std::vector<IntervalState<T>*> ordered;
  for (int s : by_a) ordered.push_back(&S[(size_t)s]);
  assemble_result<T>(ctx, A, ordered, bd.normA, out);
  out->slice_counts.assign((size_t)ns, 0);
  bool all_done = true;
  for (int s = 0; s < ns; ++s) {
    out->slice_counts[(size_t)s] = (int64_t)S[(size_t)s].lam_lock.size();
    all_done = all_done && S[(size_t)s].done;
  }
  st.max_residual = 0.0;
  for (double r : out->res) st.max_residual = std::max(st.max_residual, r);
  st.gpu_launches = ctx->launches - launches0;
  st.ms_total = std::chrono::duration<double, std::milli>(clock::now() - t_start).count();
  out->history = hist;
  out->stats = st;
  if (!all_done) throw ApfError{APF_ERR_NO_CONVERGENCE, "no convergence"};
}

void solve(apf_ctx* ctx, const apf_matrix* A, const apf_params* prm, apf_result* out) {
  if (A->dtype == APF_C128) solve_t<double2>(ctx, A, prm, out);
  else solve_t<double>(ctx, A, prm, out);
}

void solve_slices(apf_ctx* ctx, const apf_matrix* A, int nslices, const double* a, const double* b,
                  const int64_t* p, const apf_params* prm, apf_result* out) {
  if (A->dtype == APF_C128) solve_slices_t<double2>(ctx, A, nslices, a, b, p, prm, out);
  else solve_slices_t<double>(ctx, A, nslices, a, b, p, prm, out);
}

// ---- the steps one by one, on caller buffers ------------------------------------------
template <class T>
static DBuf stage_in(apf_ctx* ctx, int64_t n, int64_t p, const T* X, int64_t ldx, int64_t ld) {
  DBuf b((size_t)n * ld * sizeof(T), ctx->stream, true);
  APF_CUDA(cudaMemcpy2DAsync(b.p, ld * sizeof(T), X, ldx * sizeof(T), p * sizeof(T), n,
                             cudaMemcpyDeviceToDevice, ctx->stream));
  return b;
}

template <class T>
static void stage_out(apf_ctx* ctx, int64_t n, int64_t p, const T* X, int64_t ld, T* Y, int64_t ldy) {
  APF_CUDA(cudaMemcpy2DAsync(Y, ldy * sizeof(T), X, ld * sizeof(T), p * sizeof(T), n,
                             cudaMemcpyDeviceToDevice, ctx->stream));
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
}

template <class T>
void filter_apply_public(apf_ctx* ctx, const apf_matrix* A, const double* coef, int k, double l1,
                         double l2, int precision, const T* X, int64_t ldx, int64_t p, T* Y,
                         int64_t ldy) {
  const int64_t n = A->n, ld = block_ld(p);
  DBuf V = stage_in<T>(ctx, n, p, X, ldx, ld);
  DBuf out((size_t)n * ld * sizeof(T), ctx->stream, true);
  FilterState<T> fs;
  fs.init(ctx, A, ld, l1, l2, std::vector<double>(coef, coef + k + 1), precision);
  FilterCount fc;
  fs.apply(k, V.as<T>(), nullptr, nullptr, p, out.as<T>(), nullptr, nullptr, &fc);
  stage_out<T>(ctx, n, p, out.as<T>(), ld, Y, ldy);
}

template <class T>
void filter_apply_defect_public(apf_ctx* ctx, const apf_matrix* A, const double* coef, int k,
                                double l1, double l2, const T* V, const T* AV, const double* lam,
                                int64_t ld_in, int64_t p, T* Y, int64_t ldy) {
  const int64_t n = A->n, ld = block_ld(p);
  DBuf Vb = stage_in<T>(ctx, n, p, V, ld_in, ld);
  DBuf AVb = stage_in<T>(ctx, n, p, AV, ld_in, ld);
  DBuf out((size_t)n * ld * sizeof(T), ctx->stream, true);
  FilterState<T> fs;
  fs.init(ctx, A, ld, l1, l2, std::vector<double>(coef, coef + k + 1), APF_FILTER_F32_DEFECT);
  FilterCount fc;
  fs.apply(k, Vb.as<T>(), AVb.as<T>(), lam, p, out.as<T>(), nullptr, nullptr, &fc);
  stage_out<T>(ctx, n, p, out.as<T>(), ld, Y, ldy);
}

template <class T>
double count_estimate_public(apf_ctx* ctx, const apf_matrix* A, const double* coef, int k, double l1, double l2,
                             int precision, int64_t m, uint64_t seed) {
  const std::vector<double> c(coef, coef + k + 1);
  return count_estimates<T>(ctx, A, precision, l1, l2, {&c}, m, seed)[0];
}
template double count_estimate_public<double>(apf_ctx*, const apf_matrix*, const double*, int, double, double, int,
                                              int64_t, uint64_t);
template double count_estimate_public<double2>(apf_ctx*, const apf_matrix*, const double*, int, double, double, int,
                                               int64_t, uint64_t);

template <class T>
void spmm_public(apf_ctx* ctx, const apf_matrix* A, const T* X, int64_t ldx, int64_t p, T* Y,
                 int64_t ldy) {
  const int64_t n = A->n, ld = block_ld(p);
  DBuf Xb = stage_in<T>(ctx, n, p, X, ldx, ld);
  DBuf out((size_t)n * ld * sizeof(T), ctx->stream, true);
  spmm_plain<T>(ctx, A, Xb.as<T>(), ld, p, out.as<T>());
  stage_out<T>(ctx, n, p, out.as<T>(), ld, Y, ldy);
}

template <class T>
void cholqr2_public(apf_ctx* ctx, int64_t n, int64_t p, T* X, int64_t ldx) {
  const int64_t ld = block_ld(p);
  DBuf Xb = stage_in<T>(ctx, n, p, X, ldx, ld);
  DBuf X1((size_t)n * ld * sizeof(T), ctx->stream, true);
  SmallWork<T> sw;
  sw.init(p, ctx->stream);
  cholqr2_inplace<T>(ctx, n, p, Xb.as<T>(), X1.as<T>(), ld, sw);
  stage_out<T>(ctx, n, p, Xb.as<T>(), ld, X, ldx);
}

template <class T>
void rayleigh_ritz_public(apf_ctx* ctx, const apf_matrix* A, const T* Q, int64_t ldq, int64_t p,
                          double* w, T* V, int64_t ldv) {
  const int64_t n = A->n, ld = block_ld(p);
  DBuf Qb = stage_in<T>(ctx, n, p, Q, ldq, ld);
  DBuf AQ((size_t)n * ld * sizeof(T), ctx->stream, true);
  DBuf Vb((size_t)n * ld * sizeof(T), ctx->stream, true);
  SmallWork<T> sw;
  sw.init(p, ctx->stream);
  spmm_plain<T>(ctx, A, Qb.as<T>(), ld, p, AQ.as<T>());
  gram<T>(ctx, n, p, p, Qb.as<T>(), ld, AQ.as<T>(), ld, sw.B, p, false);
  symmetrize<T>(ctx, p, sw.B, p);
  eigh_jacobi<T>(ctx, p, sw.B, p, w, sw.U, p);
  gemm_tall<T>(ctx, n, p, p, Qb.as<T>(), ld, sw.U, p, Vb.as<T>(), ld, 1.0, 0.0, nullptr, ld, false);
  const int derr = fetch_device_error(ctx);
  if (derr == DEV_EIGH_NOCONV) throw ApfError{APF_ERR_EIGH, "eigh"};
  if (derr == DEV_BARRIER_TIMEOUT) throw ApfError{APF_ERR_TIMEOUT, "eigh barrier"};
  stage_out<T>(ctx, n, p, Vb.as<T>(), ld, V, ldv);
}

template <class T>
void residual_norms_public(apf_ctx* ctx, const apf_matrix* A, const T* V, int64_t ldv, int64_t p,
                           const double* w, double* host_out) {
  const int64_t n = A->n, ld = block_ld(p);
  DBuf Vb = stage_in<T>(ctx, n, p, V, ldv, ld);
  DBuf AV((size_t)n * ld * sizeof(T), ctx->stream, true);
  DBuf rd((size_t)p * sizeof(double), ctx->stream, false);
  spmm_plain<T>(ctx, A, Vb.as<T>(), ld, p, AV.as<T>());
  residual_norms<T>(ctx, n, p, AV.as<T>(), Vb.as<T>(), ld, w, rd.as<double>(), nullptr, 0.0);
  APF_CUDA(cudaMemcpyAsync(host_out, rd.p, (size_t)p * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
}

// Failure-path check of the two-step filter pass: one pass over the matrix's
// SELL copy (FP32, width 8, zero values) in which every step-2 item waits for
// step-1 counts of pass 1000, which the counters (zero before the launch, so
// at most 1 after it) never reach.  Every waiting CTA gives up after the
// context's wait limit, records DEV_BARRIER_TIMEOUT and leaves; the host turns
// that into APF_ERR_TIMEOUT.
void wait_probe_pair(apf_ctx* ctx, const apf_matrix* A) {
  APF_REQUIRE(A->sell_ok, APF_ERR_ARG);
  const int G = 8, VPT = 1;  // a compiled shape (kSellShapes)
  const int R = 256 / G;
  APF_REQUIRE((int64_t)R * 4 < A->n, APF_ERR_ARG);
  const int64_t n = A->n, ld = 8;
  DBuf vals((size_t)A->sell_slots * sizeof(float), ctx->stream, true);
  DBuf a((size_t)n * ld * sizeof(float), ctx->stream, true), b((size_t)n * ld * sizeof(float), ctx->stream, true);
  DBuf y((size_t)n * ld * sizeof(float), ctx->stream, true);
  const size_t segs = (size_t)((n + 8 * PAIR_SEG - 1) / (8 * PAIR_SEG) + 1) * sizeof(unsigned);
  DBuf seg(segs, ctx->stream, true);
  clenshaw_sell_pair<float, float>(ctx, G, VPT, n, A->sell_chunk_ptr, A->sell_col, vals.as<float>(), A->sell_lmax,
                                   A->sell_bw, a.as<float>(), b.as<float>(), nullptr, y.as<float>(), ld, ld,
                                   nullptr, 0.5f, nullptr, 0.25f, seg.as<unsigned>(), 1000u);
  const int e = fetch_device_error(ctx);
  if (e == DEV_BARRIER_TIMEOUT) throw ApfError{APF_ERR_TIMEOUT, "two-step filter dependency wait"};
  if (e != 0) throw ApfError{APF_ERR_CUDA, "device error in the wait probe"};
}

#define APF_INST(T)                                                                                  \
  template void filter_apply_public<T>(apf_ctx*, const apf_matrix*, const double*, int, double,     \
                                       double, int, const T*, int64_t, int64_t, T*, int64_t);       \
  template void filter_apply_defect_public<T>(apf_ctx*, const apf_matrix*, const double*, int,      \
                                              double, double, const T*, const T*, const double*,    \
                                              int64_t, int64_t, T*, int64_t);                       \
  template void spmm_public<T>(apf_ctx*, const apf_matrix*, const T*, int64_t, int64_t, T*,         \
                               int64_t);                                                            \
  template void cholqr2_public<T>(apf_ctx*, int64_t, int64_t, T*, int64_t);                         \
  template void rayleigh_ritz_public<T>(apf_ctx*, const apf_matrix*, const T*, int64_t, int64_t,    \
                                        double*, T*, int64_t);                                      \
  template void residual_norms_public<T>(apf_ctx*, const apf_matrix*, const T*, int64_t, int64_t,   \
                                         const double*, double*);
APF_INST(double)
APF_INST(double2)
#undef APF_INST

}  // namespace apf
