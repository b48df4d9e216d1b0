// The serving engine's per-request solve: Alg. 4 for one request, advanced one
// outer iteration at a time by the serving loop, with the filter recurrence
// (Alg. 2) exposed step by step so that the Clenshaw steps of every running
// request share one launch (spmm_multi.cuh).  Everything else -- bounds,
// coefficients, the subspace size of Sec. 3.4, the orthogonalisation,
// Rayleigh-Ritz, residuals, the spurious rule, locking and Alg. 3 -- is the
// single solve's code on the request's own stream, so a served request
// computes exactly what apf_solve computes for it.
#include "engine.h"
#include "solver_impl.cuh"

namespace apf {

namespace {

template <class T>
class EngineSolveT final : public EngineSolve {
  using TL = typename LowOf<T>::type;
  static constexpr int E = ScalarTraits<TL>::per16;

 public:
  EngineSolveT(apf_ctx* c, const apf_matrix* M, const apf_params* p) : A(M), prm(*p) {
    ctx = c;
    t_start = std::chrono::steady_clock::now();
    launches0 = ctx->launches;
  }

  void setup() {
    const int64_t n = A->n;
    APF_REQUIRE(prm.p >= 0 && prm.p <= n && prm.p <= APF_MAX_P, APF_ERR_ARG);
    APF_REQUIRE(prm.p > 0 || (prm.init_block == nullptr && prm.mu > 0.0 && prm.trace_probes >= 1), APF_ERR_ARG);
    APF_REQUIRE(prm.a < prm.b && prm.max_iter >= 1, APF_ERR_ARG);
    APF_REQUIRE(prm.filter_precision >= APF_FILTER_F64 && prm.filter_precision <= APF_FILTER_F32_DEFECT,
                APF_ERR_ARG);
    bd = setup_bounds(ctx, A, &prm);
    S.setup_filter(&prm, prm.a, prm.b, bd.l1, bd.l2);
    int64_t p = prm.p;
    if (p == 0) {
      st.trace_estimate = count_estimates<T>(ctx, A, prm.filter_precision, bd.l1, bd.l2, {&S.coef},
                                             prm.trace_probes, prm.seed)[0];
      p = subspace_size(st.trace_estimate, prm.mu, n);
    }
    st.p_used = p;
    sw.init(p, ctx->stream);
    S.init_block(ctx, A, &prm, p, 1u, sw);
    st.k1 = S.k1;
    st.k_max = S.kmax;
    st.lambda_min = bd.lmin;
    st.lambda_max = bd.lmax;
    st.norm_a = bd.normA;
    fs.init(ctx, A, S.ld, bd.l1, bd.l2, S.coef, prm.filter_precision);
    fs.graphs_on = prm.filter_graphs != 0;  // for the iterations it filters on its own
    APF_CUDA(cudaStreamSynchronize(ctx->stream));
    st.ms_setup = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  }

  void begin_iteration() override {
    ev = IterEv{evp.get(), evp.get(), evp.get(), evp.get(), evp.get(), evp.get()};
    iev.push_back(ev);
    APF_CUDA(cudaEventRecord(ev.e0, ctx->stream));
    APF_CUDA(cudaEventRecord(ev.f0, ctx->stream));
    k = S.ki;
    const int64_t n = A->n, p = S.pa, ld = S.ld;
    defect = S.have_ritz && prm.filter_precision == APF_FILTER_F32_DEFECT;
    // batch the steps of problems too small to fill the GPU alone (fewer tiles
    // of the batched step than eight per SM); larger ones, FP64 filters and
    // matrices without a SELL copy filter on their own stream, concurrently
    const int64_t tiles = ((n + 31) / 32) * (((p + E - 1) / E + 15) / 16);
    batched_ = prm.filter_precision != APF_FILTER_F64 && A->sell_ok && tiles < 8LL * ctx->num_sms;
    nsteps = 0;
    result = nullptr;
    if (!batched_) {  // this request filters on its own stream
      fs.apply(k, S.Vh.template as<T>(), defect ? S.AVh.template as<T>() : nullptr, defect ? S.w : nullptr, p,
               S.X.template as<T>(), nullptr, nullptr, &fc);
      return;
    }
    TL* B1 = fs.B1.template as<TL>();
    TL* Yr = fs.Y32.template as<TL>();
    b1 = B1;
    b2 = fs.B2.template as<TL>();
    if (defect) {
      // R_hat = l1 (A V - V diag(lam)) in FP32 and the per-column coefficients
      DBuf scratch((size_t)p * sizeof(double), ctx->stream, false);
      residual_norms<T>(ctx, n, p, S.AVh.template as<T>(), S.Vh.template as<T>(), ld, S.w, scratch.as<double>(), Yr,
                        bd.l1);
      defect_coefficients(ctx, p, ld, k, fs.coef_dev.template as<double>(), S.w, bd.l1, bd.l2,
                          fs.F.template as<float>(), fs.rho.template as<double>());
      if (k == 1) {
        scale_columns<TL>(ctx, n, p, fs.F.template as<float>(), Yr, ld, B1);
        result = B1;
      } else if (k >= 2) {
        scale_columns<TL>(ctx, n, p, fs.F.template as<float>() + (int64_t)(k - 1) * ld, Yr, ld, B1);
        nsteps = k - 1;
      }
    } else {
      cast_block_rows<T, TL>(ctx, n, p, S.Vh.template as<T>(), ld, Yr, ld, nullptr);
      scale_block<TL>(ctx, n, p, fs.a[(size_t)k], Yr, ld, B1, ld);  // b_k = a_k Y
      if (k == 0) result = B1;
      else nsteps = k;
    }
    P1 = B1;
    P2 = nullptr;
  }

  bool batched() const override { return batched_; }
  bool is_complex() const override { return ScalarTraits<T>::is_complex; }
  int steps() const override { return batched_ ? nsteps : 0; }

  void step_desc(int g, MultiDesc* d) override {
    const int j = g;
    const int64_t p = S.pa, ld = S.ld;
    TL* other = P1 == b1 ? b2 : b1;
    TL* out = P2 ? P2 : other;
    d->chunk_ptr = A->sell_chunk_ptr;
    d->scol = A->sell_col;
    d->sval = fs.Asell32.p;
    d->W = P1;
    d->Vin = P2;
    d->Y = fs.Y32.p;
    d->Out = out;
    d->coef_col = defect ? fs.F.template as<float>() + (int64_t)j * ld : nullptr;
    d->coef_scalar = defect ? 0.0f : (float)fs.a[(size_t)j];
    d->alpha = j == 0 ? 1.0f : 2.0f;
    d->n = A->n;
    d->ld = ld;
    d->nvec = (int)((p + E - 1) / E);
    d->lmax = A->sell_lmax;
    const double b = step_bytes(A->n, A->nnz, p, sizeof(TL), sizeof(TL), P2 != nullptr, true);
    fc.steps += 1;
    fc.launches += 1;
    fc.bytes += b;
    fc.step_bytes += b;
    P2 = P1;
    P1 = out;
    if (j == 0) result = P1;
  }

  void end_iteration() override {
    const int64_t n = A->n, p = S.pa, ld = S.ld;
    if (batched_) {
      if (defect)
        defect_combine<T>(ctx, n, p, S.Vh.template as<T>(), ld, fs.rho.template as<double>(), result, ld,
                          S.X.template as<T>(), ld, nullptr);
      else
        cast_block_rows<TL, T>(ctx, n, p, result, ld, S.X.template as<T>(), ld, nullptr);
    }
    APF_CUDA(cudaEventRecord(ev.f1, ctx->stream));
    st.spmv_columns += (int64_t)k * p + 2 * p;
    deg_sum += k;
    ++iters;
    APF_CUDA(cudaEventRecord(ev.e1, ctx->stream));
    S.orth(ctx, A, sw, prm.gram_tensor_cores != 0);
    APF_CUDA(cudaEventRecord(ev.e2, ctx->stream));
  }

  void check() override {
    check_device_after_rr(ctx);
    S.check(ctx, A, &prm, bd.l1, bd.l2, bd.normA);
    APF_CUDA(cudaEventRecord(ev.e3, ctx->stream));
    hist.insert(hist.end(), S.rec.begin(), S.rec.end());
    if (S.done) {
      status = APF_OK;
      finished_ = true;
    } else if (S.pa == 0 || iters >= prm.max_iter) {
      finished_ = true;
    }
  }

  bool finished() const override { return finished_; }

  apf_result* take_result(apf_status* out_status) override {
    auto* out = new apf_result();
    try {
      finish_stats(ctx, iev, fc, iters, deg_sum, &st);
      assemble_result<T>(ctx, A, {&S}, bd.normA, out);
    } catch (...) {
      delete out;
      throw;
    }
    st.max_residual = 0.0;
    for (double r : out->res) st.max_residual = std::max(st.max_residual, r);
    st.gpu_launches = ctx->launches - launches0;
    st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    out->history = hist;
    out->stats = st;
    *out_status = status;
    return out;
  }

 private:
  const apf_matrix* A;
  apf_params prm;
  Bounds bd{};
  IntervalState<T> S;
  FilterState<T> fs;
  SmallWork<T> sw;
  apf_stats st{};
  FilterCount fc;
  EventPool evp;
  std::vector<IterEv> iev;
  IterEv ev{};
  std::vector<double> hist;
  std::chrono::steady_clock::time_point t_start;
  int64_t launches0 = 0;
  double deg_sum = 0.0;
  int iters = 0;
  apf_status status = APF_ERR_NO_CONVERGENCE;
  bool finished_ = false;
  // this iteration's recurrence
  int k = 0, nsteps = 0;
  bool defect = false, batched_ = false;
  TL *b1 = nullptr, *b2 = nullptr, *P1 = nullptr, *P2 = nullptr, *result = nullptr;
};

}  // namespace

std::unique_ptr<EngineSolve> engine_start(apf_ctx* ctx, const apf_matrix* A, const apf_params* prm) {
  if (A->dtype == APF_C128) {
    auto s = std::make_unique<EngineSolveT<double2>>(ctx, A, prm);
    s->setup();
    return s;
  }
  auto s = std::make_unique<EngineSolveT<double>>(ctx, A, prm);
  s->setup();
  return s;
}

void engine_step_launch(apf_ctx* ctx, bool cplx, MultiArgs& a) {
  if (cplx) clenshaw_multi_launch<float2>(ctx, a);
  else clenshaw_multi_launch<float>(ctx, a);
}

}  // namespace apf
