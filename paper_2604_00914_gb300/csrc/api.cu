// The C ABI of include/apf.h: argument checks, object lifetimes and the
// exception-to-status boundary.  Matrix ingest validates CSR structure, adds
// missing diagonal entries, checks A = A^H and uploads the arrays.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "host_math.h"
#include "solver.h"


#define APF_TRY(ctxp)                                            \
  try {
#define APF_CATCH(ctxp)                                          \
  }                                                              \
  catch (const ApfError& e) {                                    \
    if (ctxp) (ctxp)->last_error = e.what;                       \
    return e.status;                                             \
  }                                                              \
  catch (...) {                                                  \
    return APF_ERR_CUDA;                                         \
  }                                                              \
  return APF_OK;

static void bind(apf_ctx* ctx) { APF_CUDA(cudaSetDevice(ctx->device)); }

extern "C" {

const char* apf_status_string(int s) {
  switch (s) {
    case APF_OK: return "ok";
    case APF_ERR_ARG: return "invalid argument";
    case APF_ERR_OOM: return "device out of memory";
    case APF_ERR_CUDA: return "CUDA error";
    case APF_ERR_NOT_HERMITIAN: return "matrix is not Hermitian";
    case APF_ERR_CHOL: return "Cholesky QR breakdown";
    case APF_ERR_NO_CONVERGENCE: return "no convergence within max_iter";
    case APF_ERR_EIGH: return "small eigensolver did not converge";
    case APF_ERR_TIMEOUT: return "device wait timed out";
    case APF_ERR_NOT_READY: return "no data";
    default: return "unknown status";
  }
}

const char* apf_last_error_message(const apf_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

apf_status apf_create(apf_ctx** out, int device, void* cuda_stream) {
  if (!out) return APF_ERR_ARG;
  apf_ctx* ctx = new apf_ctx();
  try {
    int ndev = 0;
    APF_CUDA(cudaGetDeviceCount(&ndev));
    APF_REQUIRE(device >= 0 && device < ndev, APF_ERR_ARG);
    ctx->device = device;
    APF_CUDA(cudaSetDevice(device));
    APF_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
    if (cuda_stream) {
      ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      APF_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
      ctx->own_stream = true;
    }
    APF_CUDA(cudaMalloc(&ctx->d_err, sizeof(int)));
    APF_CUDA(cudaMalloc(&ctx->d_bar, 4 * sizeof(unsigned)));
    APF_CUDA(cudaMalloc(&ctx->d_counters, 64 * sizeof(unsigned)));
    APF_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    APF_CUDA(cudaMemsetAsync(ctx->d_bar, 0, 4 * sizeof(unsigned), ctx->stream));
    APF_CUDA(cudaStreamSynchronize(ctx->stream));
  } catch (const ApfError& e) {
    apf_destroy(ctx);
    return e.status;
  }
  *out = ctx;
  return APF_OK;
}

apf_status apf_destroy(apf_ctx* ctx) {
  if (!ctx) return APF_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->d_bar) cudaFree(ctx->d_bar);
  if (ctx->d_counters) cudaFree(ctx->d_counters);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return APF_OK;
}

int64_t apf_launch_count(const apf_ctx* ctx) { return ctx ? ctx->launches : 0; }

apf_status apf_set_wait_limit(apf_ctx* ctx, int64_t ns) {
  if (!ctx || ns < 0 || ns > 60000000000LL) return APF_ERR_ARG;
  ctx->wait_limit_ns = (uint64_t)ns;
  return APF_OK;
}

apf_status apf_wait_probe(apf_ctx* ctx, const apf_matrix* A, int32_t which) {
  if (!ctx || (which != 0 && which != 1) || (which == 0 && (!A || A->ctx != ctx))) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (which == 0) apf::wait_probe_pair(ctx, A);
  else apf::wait_probe_barrier(ctx);
  APF_CATCH(ctx)
}

void apf_params_default(apf_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->a = 0.0;
  p->b = 0.0;
  p->p = 0;
  p->k_fixed = 0;
  p->damping = APF_DAMP_LANCZOS_M;
  p->C = 1.4;
  p->k_ratio = 2.5;
  p->m_d = 0.5;
  p->tau_a = 1e-3;
  p->tau_c = 1e-10;
  p->max_iter = 50;
  p->lanczos_steps = 40;
  p->bound_pad = 0.01;
  p->filter_precision = APF_FILTER_F64;
  p->spurious_rule = 1;
  p->seed = 20260401ull;
  p->init_block = nullptr;
  p->init_on_device = 0;
  p->max_degree_cap = 100000;
  p->mu = 1.8;
  p->trace_probes = 32;
  p->filter_graphs = 1;
  p->gram_tensor_cores = 1;
}

}  // extern "C"

// ---- matrix ingest ---------------------------------------------------------------

// Reverse Cuthill-McKee ordering (Cuthill and McKee 1969; George 1971):
// breadth-first search from a pseudo-peripheral vertex of each component,
// neighbours taken in increasing degree, the visit order reversed.
// Returns new -> old.
static std::vector<int32_t> rcm_order(int64_t n, const std::vector<int64_t>& rp,
                                      const std::vector<int32_t>& ci) {
  std::vector<int32_t> order;
  order.reserve((size_t)n);
  std::vector<char> seen((size_t)n, 0);
  std::vector<int32_t> level((size_t)n, -1), q((size_t)n), nb;
  auto deg = [&](int64_t v) { return rp[(size_t)v + 1] - rp[(size_t)v]; };
  // last level of a BFS from s, restricted to s's component
  auto bfs_far = [&](int32_t s, int* depth) {
    std::vector<int32_t> touched;
    int64_t h = 0, t = 0;
    q[(size_t)t++] = s;
    level[(size_t)s] = 0;
    touched.push_back(s);
    int32_t best = s;
    while (h < t) {
      const int32_t u = q[(size_t)h++];
      for (int64_t e = rp[(size_t)u]; e < rp[(size_t)u + 1]; ++e) {
        const int32_t v = ci[(size_t)e];
        if (level[(size_t)v] < 0) {
          level[(size_t)v] = level[(size_t)u] + 1;
          q[(size_t)t++] = v;
          touched.push_back(v);
        }
      }
    }
    const int maxl = level[(size_t)q[(size_t)t - 1]];
    for (int32_t v : touched)
      if (level[(size_t)v] == maxl && deg(v) < deg(best)) best = v;
    if (level[(size_t)best] != maxl) best = q[(size_t)t - 1];
    *depth = maxl;
    for (int32_t v : touched) level[(size_t)v] = -1;
    return best;
  };
  for (int64_t s0 = 0; s0 < n; ++s0) {
    if (seen[(size_t)s0]) continue;
    int32_t start = (int32_t)s0;
    int depth = -1;
    for (int it = 0; it < 3; ++it) {
      int d2 = 0;
      const int32_t far = bfs_far(start, &d2);
      if (d2 <= depth) break;
      depth = d2;
      start = far;
    }
    int64_t h = (int64_t)order.size();
    order.push_back(start);
    seen[(size_t)start] = 1;
    while (h < (int64_t)order.size()) {
      const int32_t u = order[(size_t)h++];
      nb.clear();
      for (int64_t e = rp[(size_t)u]; e < rp[(size_t)u + 1]; ++e) {
        const int32_t v = ci[(size_t)e];
        if (!seen[(size_t)v]) {
          seen[(size_t)v] = 1;
          nb.push_back(v);
        }
      }
      std::stable_sort(nb.begin(), nb.end(), [&](int32_t x, int32_t y) { return deg(x) < deg(y); });
      order.insert(order.end(), nb.begin(), nb.end());
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

template <class V>
static void ingest_csr(apf_ctx* ctx, int64_t n, const std::vector<int64_t>& rp_in,
                       const std::vector<int32_t>& ci_in, const std::vector<V>& v_in, int dtype,
                       apf_matrix** out) {
  const int64_t nnz_in = (int64_t)ci_in.size();
  APF_REQUIRE(rp_in.size() == (size_t)n + 1 && rp_in[0] == 0 && rp_in[(size_t)n] == nnz_in,
              APF_ERR_ARG);
  for (int64_t i = 0; i < n; ++i) APF_REQUIRE(rp_in[(size_t)i + 1] >= rp_in[(size_t)i], APF_ERR_ARG);
  for (int32_t c : ci_in) APF_REQUIRE(c >= 0 && (int64_t)c < n, APF_ERR_ARG);
  // rows sorted by column, duplicates summed, diagonal present
  std::vector<int64_t> rp((size_t)n + 1, 0);
  std::vector<int32_t> ci;
  std::vector<V> vv;
  ci.reserve((size_t)nnz_in + (size_t)n);
  vv.reserve((size_t)nnz_in + (size_t)n);
  std::vector<std::pair<int32_t, V>> row;
  double amax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    row.clear();
    bool has_diag = false;
    for (int64_t e = rp_in[(size_t)i]; e < rp_in[(size_t)i + 1]; ++e) {
      row.emplace_back(ci_in[(size_t)e], v_in[(size_t)e]);
      if (ci_in[(size_t)e] == i) has_diag = true;
      amax = std::max(amax, (double)std::abs(v_in[(size_t)e]));
    }
    if (!has_diag) row.emplace_back((int32_t)i, V(0));
    std::sort(row.begin(), row.end(), [](const std::pair<int32_t, V>& a, const std::pair<int32_t, V>& b) {
      return a.first < b.first;
    });
    for (size_t t = 0; t < row.size(); ++t) {
      if (!ci.empty() && (int64_t)ci.size() > rp[(size_t)i] && ci.back() == row[t].first) {
        vv.back() += row[t].second;
      } else {
        ci.push_back(row[t].first);
        vv.push_back(row[t].second);
      }
    }
    rp[(size_t)i + 1] = (int64_t)ci.size();
  }
  for (const V& x : vv) APF_REQUIRE(std::isfinite(std::abs(x)), APF_ERR_ARG);
  // A = A^H within a relative tolerance
  const double tol = 1e-12 * (amax > 0 ? amax : 1.0);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t e = rp[(size_t)i]; e < rp[(size_t)i + 1]; ++e) {
      const int32_t j = ci[(size_t)e];
      const auto b = ci.begin() + rp[(size_t)j], en = ci.begin() + rp[(size_t)j + 1];
      const auto it = std::lower_bound(b, en, (int32_t)i);
      V mirror = V(0);
      if (it != en && *it == i) mirror = vv[(size_t)(it - ci.begin())];
      if (std::abs(vv[(size_t)e] - std::conj(mirror)) > tol) throw ApfError{APF_ERR_NOT_HERMITIAN, "A != A^H"};
    }
  }
  apf_matrix* A = new apf_matrix();
  A->ctx = ctx;
  A->n = n;
  A->nnz = (int64_t)ci.size();
  A->dtype = dtype;
  // Row order for the filter: the natural one, or reverse Cuthill-McKee when
  // that at least halves the bandwidth max |i - j| (a small bandwidth lets the
  // filter run two steps per pass out of L2).
  int64_t bw0 = 0;
  constexpr int kNearMax = 16;
  int64_t near[kNearMax + 1] = {0};  // entries at each distance |i - j| <= kNearMax
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rp[(size_t)i]; e < rp[(size_t)i + 1]; ++e) {
      const int64_t dist = std::abs((int64_t)ci[(size_t)e] - i);
      bw0 = std::max<int64_t>(bw0, dist);
      if (dist <= kNearMax) ++near[dist];
    }
  // Near-row reach of the column-tiled step: a CTA of 32 rows that stages rows
  // r0 - H .. r0 + 32 + H of W reads the entries within H of the diagonal from
  // shared memory at the cost of (32 + 2 H) / 32 staged rows per row; keep the
  // H in {1, 2, 4, 8, 16} that saves the most row reads, if it saves at least
  // one per row.
  int halo = 0;
  {
    double best = 1.0;
    int64_t within = near[0];
    for (int h = 1; h <= kNearMax; ++h) {
      within += near[h];
      if ((h & (h - 1)) != 0) continue;
      const double saved = (n > 0 ? (double)within / (double)n : 0.0) - (32.0 + 2.0 * h) / 32.0;
      if (saved > best + 1e-12) { best = saved; halo = h; }
    }
  }
  std::vector<int32_t> perm, iperm;  // perm: new -> old, iperm: old -> new
  int64_t bw = bw0;
  if (bw0 > 4096 && n < INT32_MAX) {
    perm = rcm_order(n, rp, ci);
    iperm.assign((size_t)n, 0);
    for (int64_t r = 0; r < n; ++r) iperm[(size_t)perm[(size_t)r]] = (int32_t)r;
    int64_t bw1 = 0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t e = rp[(size_t)i]; e < rp[(size_t)i + 1]; ++e)
        bw1 = std::max<int64_t>(bw1, std::abs((int64_t)iperm[(size_t)ci[(size_t)e]] - (int64_t)iperm[(size_t)i]));
    if (2 * bw1 <= bw0) bw = bw1;
    else { perm.clear(); iperm.clear(); }
  }
  const bool permuted = !perm.empty();
  // SELL-8 structures (chunks of 8 consecutive rows padded to their longest
  // row), each row's entries in CSR order so that every form sums in the same
  // order: one in the natural row order, and one in the permuted order when a
  // permutation was found.  Used when padding costs at most half the entries.
  struct Sell {
    std::vector<int64_t> cptr;
    std::vector<int32_t> col, src;
    int lmax = 0;
    int64_t slots = 0;
  };
  const int CH = 8;
  const int64_t nchunks = (n + CH - 1) / CH;
  auto build_sell = [&](bool use_perm, Sell& S) {
    auto old_row = [&](int64_t r) { return use_perm ? (int64_t)perm[(size_t)r] : r; };
    auto new_col = [&](int32_t c) { return use_perm ? iperm[(size_t)c] : c; };
    S.cptr.assign((size_t)nchunks + 1, 0);
    for (int64_t c = 0; c < nchunks; ++c) {
      int64_t L = 0;
      for (int64_t r = c * CH; r < std::min<int64_t>(n, (c + 1) * CH); ++r) {
        const int64_t o = old_row(r);
        L = std::max<int64_t>(L, rp[(size_t)o + 1] - rp[(size_t)o]);
      }
      S.lmax = std::max<int>(S.lmax, (int)L);
      S.cptr[(size_t)c + 1] = S.cptr[(size_t)c] + L * CH;
    }
    S.slots = S.cptr[(size_t)nchunks];
    S.col.assign((size_t)S.slots, 0);
    S.src.assign((size_t)S.slots, -1);
    for (int64_t c = 0; c < nchunks; ++c) {
      const int64_t L = (S.cptr[(size_t)c + 1] - S.cptr[(size_t)c]) / CH;
      for (int64_t r = c * CH; r < (c + 1) * CH; ++r) {
        const int64_t o = r < n ? old_row(r) : -1;
        const int64_t len = o >= 0 ? rp[(size_t)o + 1] - rp[(size_t)o] : 0;
        for (int64_t t = 0; t < L; ++t) {
          const size_t sl = (size_t)(S.cptr[(size_t)c] + t * CH + (r - c * CH));
          if (t < len) {
            S.col[sl] = new_col(ci[(size_t)(rp[(size_t)o] + t)]);
            S.src[sl] = (int32_t)(rp[(size_t)o] + t);
          } else {
            S.col[sl] = (int32_t)(r < n ? r : 0);  // padding: the row itself, value 0
          }
        }
      }
    }
  };
  int64_t slots0 = 0;
  {
    for (int64_t c = 0; c < nchunks; ++c) {
      int64_t L = 0;
      for (int64_t r = c * CH; r < std::min<int64_t>(n, (c + 1) * CH); ++r)
        L = std::max<int64_t>(L, rp[(size_t)r + 1] - rp[(size_t)r]);
      slots0 += L * CH;
    }
  }
  const bool sell_ok = slots0 <= (int64_t)(1.5 * (double)A->nnz) && A->nnz < INT32_MAX && slots0 < INT32_MAX;
  Sell nat, prm;
  if (sell_ok) {
    build_sell(false, nat);
    if (permuted) {
      build_sell(true, prm);
      if (prm.slots > (int64_t)(1.5 * (double)A->nnz) || prm.slots >= INT32_MAX) {
        perm.clear();
        iperm.clear();
      }
    }
  }
  const bool have_perm = sell_ok && !perm.empty();
  try {
    APF_CUDA(cudaMalloc(&A->rowptr, rp.size() * sizeof(int64_t)));
    APF_CUDA(cudaMalloc(&A->colidx, std::max<size_t>(ci.size(), 1) * sizeof(int32_t)));
    APF_CUDA(cudaMalloc(&A->vals, std::max<size_t>(vv.size(), 1) * sizeof(V)));
    APF_CUDA(cudaMemcpyAsync(A->rowptr, rp.data(), rp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
    APF_CUDA(cudaMemcpyAsync(A->colidx, ci.data(), ci.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    APF_CUDA(cudaMemcpyAsync(A->vals, vv.data(), vv.size() * sizeof(V), cudaMemcpyHostToDevice, ctx->stream));
    if (sell_ok) {
      A->sell_ok = true;
      A->sell_lmax = nat.lmax;
      A->sell_slots = nat.slots;
      A->sell_bw = bw0;
      A->sell_halo = halo;
      APF_CUDA(cudaMalloc(&A->sell_chunk_ptr, nat.cptr.size() * sizeof(int64_t)));
      APF_CUDA(cudaMalloc(&A->sell_col, std::max<size_t>(nat.col.size(), 1) * sizeof(int32_t)));
      APF_CUDA(cudaMalloc(&A->sell_src, std::max<size_t>(nat.src.size(), 1) * sizeof(int32_t)));
      APF_CUDA(cudaMemcpyAsync(A->sell_chunk_ptr, nat.cptr.data(), nat.cptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
      APF_CUDA(cudaMemcpyAsync(A->sell_col, nat.col.data(), nat.col.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
      APF_CUDA(cudaMemcpyAsync(A->sell_src, nat.src.data(), nat.src.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    }
    if (have_perm) {
      A->psell_lmax = prm.lmax;
      A->psell_slots = prm.slots;
      A->psell_bw = bw;
      APF_CUDA(cudaMalloc(&A->perm, perm.size() * sizeof(int32_t)));
      APF_CUDA(cudaMalloc(&A->iperm, iperm.size() * sizeof(int32_t)));
      APF_CUDA(cudaMemcpyAsync(A->perm, perm.data(), perm.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
      APF_CUDA(cudaMemcpyAsync(A->iperm, iperm.data(), iperm.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
      APF_CUDA(cudaMalloc(&A->psell_chunk_ptr, prm.cptr.size() * sizeof(int64_t)));
      APF_CUDA(cudaMalloc(&A->psell_col, std::max<size_t>(prm.col.size(), 1) * sizeof(int32_t)));
      APF_CUDA(cudaMalloc(&A->psell_src, std::max<size_t>(prm.src.size(), 1) * sizeof(int32_t)));
      APF_CUDA(cudaMemcpyAsync(A->psell_chunk_ptr, prm.cptr.data(), prm.cptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
      APF_CUDA(cudaMemcpyAsync(A->psell_col, prm.col.data(), prm.col.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
      APF_CUDA(cudaMemcpyAsync(A->psell_src, prm.src.data(), prm.src.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    }
    if (dtype == APF_C128)
      apf::gershgorin<double2>(ctx, n, A->rowptr, A->colidx, static_cast<const double2*>(A->vals), &A->gersh_lo, &A->gersh_hi);
    else
      apf::gershgorin<double>(ctx, n, A->rowptr, A->colidx, static_cast<const double*>(A->vals), &A->gersh_lo, &A->gersh_hi);
  } catch (...) {
    apf_matrix_destroy(A);
    throw;
  }
  *out = A;
}

template <class V>
static std::vector<V> fetch_vals(const void* vals, int64_t nnz, bool on_device) {
  std::vector<V> v((size_t)nnz);
  if (nnz == 0) return v;
  if (on_device) APF_CUDA(cudaMemcpy(v.data(), vals, (size_t)nnz * sizeof(V), cudaMemcpyDeviceToHost));
  else memcpy(v.data(), vals, (size_t)nnz * sizeof(V));
  return v;
}

extern "C" {

apf_status apf_matrix_create_csr(apf_ctx* ctx, int64_t n, int64_t nnz, const int64_t* rowptr,
                                 const int32_t* colidx, const void* vals, int32_t dtype,
                                 int32_t on_device, apf_matrix** out) {
  if (!ctx || !out || n < 1 || nnz < 0 || !rowptr || (nnz > 0 && (!colidx || !vals))) return APF_ERR_ARG;
  if (dtype != APF_R64 && dtype != APF_C128) return APF_ERR_ARG;
  if (n > INT32_MAX) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  std::vector<int64_t> rp((size_t)n + 1);
  std::vector<int32_t> ci((size_t)nnz);
  if (on_device) {
    APF_CUDA(cudaMemcpy(rp.data(), rowptr, rp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (nnz) APF_CUDA(cudaMemcpy(ci.data(), colidx, ci.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
  } else {
    memcpy(rp.data(), rowptr, rp.size() * sizeof(int64_t));
    if (nnz) memcpy(ci.data(), colidx, ci.size() * sizeof(int32_t));
  }
  if (dtype == APF_C128)
    ingest_csr<std::complex<double>>(ctx, n, rp, ci, fetch_vals<std::complex<double>>(vals, nnz, on_device), dtype, out);
  else
    ingest_csr<double>(ctx, n, rp, ci, fetch_vals<double>(vals, nnz, on_device), dtype, out);
  APF_CATCH(ctx)
}

}  // extern "C"

template <class V>
static void sell_to_csr(int64_t n, int32_t C, const int64_t* perm, const int64_t* chunk_ptr,
                        const int32_t* chunk_len, const int32_t* colidx, const V* vals,
                        std::vector<int64_t>& rp, std::vector<int32_t>& ci, std::vector<V>& vv) {
  const int64_t nchunks = (n + C - 1) / C;
  std::vector<std::vector<std::pair<int32_t, V>>> rows((size_t)n);
  for (int64_t c = 0; c < nchunks; ++c) {
    APF_REQUIRE(chunk_len[c] >= 0, APF_ERR_ARG);
    for (int32_t r = 0; r < C; ++r) {
      const int64_t pos = c * C + r;
      if (pos >= n) break;
      const int64_t row = perm[pos];
      APF_REQUIRE(row >= 0 && row < n, APF_ERR_ARG);
      for (int32_t t = 0; t < chunk_len[c]; ++t) {
        const int64_t e = chunk_ptr[c] + (int64_t)t * C + r;
        const V v = vals[e];
        if (v == V(0)) continue;  // padding (and explicit zeros) carry nothing
        APF_REQUIRE(colidx[e] >= 0 && colidx[e] < n, APF_ERR_ARG);
        rows[(size_t)row].emplace_back(colidx[e], v);
      }
    }
  }
  rp.assign((size_t)n + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    for (auto& pr : rows[(size_t)i]) {
      ci.push_back(pr.first);
      vv.push_back(pr.second);
    }
    rp[(size_t)i + 1] = (int64_t)ci.size();
  }
}

extern "C" {

apf_status apf_matrix_create_sell(apf_ctx* ctx, int64_t n, int32_t C, int32_t sigma,
                                  const int64_t* perm, const int64_t* chunk_ptr,
                                  const int32_t* chunk_len, const int32_t* colidx,
                                  const void* vals, int32_t dtype, apf_matrix** out) {
  if (!ctx || !out || n < 1 || C < 1 || sigma < 1 || !perm || !chunk_ptr || !chunk_len) return APF_ERR_ARG;
  if (dtype != APF_R64 && dtype != APF_C128) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  if (dtype == APF_C128) {
    std::vector<std::complex<double>> vv;
    sell_to_csr<std::complex<double>>(n, C, perm, chunk_ptr, chunk_len, colidx,
                                      static_cast<const std::complex<double>*>(vals), rp, ci, vv);
    ingest_csr<std::complex<double>>(ctx, n, rp, ci, vv, dtype, out);
  } else {
    std::vector<double> vv;
    sell_to_csr<double>(n, C, perm, chunk_ptr, chunk_len, colidx, static_cast<const double*>(vals), rp, ci, vv);
    ingest_csr<double>(ctx, n, rp, ci, vv, dtype, out);
  }
  APF_CATCH(ctx)
}

apf_status apf_matrix_destroy(apf_matrix* A) {
  if (!A) return APF_OK;
  if (A->ctx) {
    cudaSetDevice(A->ctx->device);
    cudaStreamSynchronize(A->ctx->stream);
  }
  if (A->rowptr) cudaFree(A->rowptr);
  if (A->colidx) cudaFree(A->colidx);
  if (A->vals) cudaFree(A->vals);
  if (A->sell_chunk_ptr) cudaFree(A->sell_chunk_ptr);
  if (A->sell_col) cudaFree(A->sell_col);
  if (A->sell_src) cudaFree(A->sell_src);
  if (A->perm) cudaFree(A->perm);
  if (A->iperm) cudaFree(A->iperm);
  if (A->psell_chunk_ptr) cudaFree(A->psell_chunk_ptr);
  if (A->psell_col) cudaFree(A->psell_col);
  if (A->psell_src) cudaFree(A->psell_src);
  delete A;
  return APF_OK;
}

apf_status apf_matrix_info(const apf_matrix* A, int64_t* n, int64_t* nnz, int32_t* dtype) {
  if (!A) return APF_ERR_ARG;
  if (n) *n = A->n;
  if (nnz) *nnz = A->nnz;
  if (dtype) *dtype = A->dtype;
  return APF_OK;
}

// ---- solve and results --------------------------------------------------------------
apf_status apf_solve(apf_ctx* ctx, const apf_matrix* A, const apf_params* params, apf_result** out) {
  if (!ctx || !A || !params || !out || A->ctx != ctx) return APF_ERR_ARG;
  apf_result* r = new apf_result();
  try {
    bind(ctx);
    apf::solve(ctx, A, params, r);
  } catch (const ApfError& e) {
    ctx->last_error = e.what;
    if (e.status == APF_ERR_NO_CONVERGENCE) {
      *out = r;
      return e.status;
    }
    delete r;
    cudaStreamSynchronize(ctx->stream);
    return e.status;
  } catch (...) {
    delete r;
    return APF_ERR_CUDA;
  }
  *out = r;
  return APF_OK;
}

apf_status apf_solve_slices(apf_ctx* ctx, const apf_matrix* A, int32_t nslices, const double* a,
                            const double* b, const int64_t* p, const apf_params* params, apf_result** out) {
  if (!ctx || !A || !params || !out || A->ctx != ctx || nslices < 1 || !a || !b || !p) return APF_ERR_ARG;
  apf_result* r = new apf_result();
  try {
    bind(ctx);
    apf::solve_slices(ctx, A, nslices, a, b, p, params, r);
  } catch (const ApfError& e) {
    ctx->last_error = e.what;
    if (e.status == APF_ERR_NO_CONVERGENCE) {
      *out = r;
      return e.status;
    }
    delete r;
    cudaStreamSynchronize(ctx->stream);
    return e.status;
  } catch (...) {
    delete r;
    return APF_ERR_CUDA;
  }
  *out = r;
  return APF_OK;
}

apf_status apf_result_slice_counts(const apf_result* r, int32_t nslices, int64_t* counts) {
  if (!r || !counts || nslices < 1 || (size_t)nslices != r->slice_counts.size()) return APF_ERR_ARG;
  memcpy(counts, r->slice_counts.data(), (size_t)nslices * sizeof(int64_t));
  return APF_OK;
}

apf_status apf_matrix_set_filter_kernel(apf_matrix* A, int32_t kind, int32_t G, int32_t VPT) {
  if (!A || kind < 0 || kind > 5 || G < 0 || VPT < 0) return APF_ERR_ARG;
  A->pin_kind = kind;
  A->pin_G = G;
  A->pin_VPT = VPT;
  A->tune_cache.clear();
  return APF_OK;
}

apf_status apf_result_count(const apf_result* r, int64_t* e) {
  if (!r || !e) return APF_ERR_ARG;
  *e = r->e;
  return APF_OK;
}

apf_status apf_result_eigvals(const apf_result* r, double* host_out) {
  if (!r || (!host_out && r->e > 0)) return APF_ERR_ARG;
  if (r->e) memcpy(host_out, r->lam.data(), (size_t)r->e * sizeof(double));
  return APF_OK;
}

apf_status apf_result_residuals(const apf_result* r, double* host_out) {
  if (!r || (!host_out && r->e > 0)) return APF_ERR_ARG;
  if (r->e) memcpy(host_out, r->res.data(), (size_t)r->e * sizeof(double));
  return APF_OK;
}

apf_status apf_result_eigvecs(const apf_result* r, void* out, int64_t ld, int32_t out_on_device) {
  if (!r || ld < r->n || (!out && r->e > 0)) return APF_ERR_ARG;
  if (r->e == 0) return APF_OK;
  apf_ctx* ctx = r->ctx;
  APF_TRY(ctx)
  bind(ctx);
  const size_t es = r->dtype == APF_C128 ? 16 : 8;
  apf::DBuf tmp;
  void* dst = out;
  if (!out_on_device) {
    tmp.alloc((size_t)ld * r->e * es, ctx->stream, false);
    dst = tmp.p;
  }
  if (r->dtype == APF_C128)
    apf::to_col_major<double2>(ctx, r->n, r->e, r->vecs.as<double2>(), r->lde, static_cast<double2*>(dst), ld);
  else
    apf::to_col_major<double>(ctx, r->n, r->e, r->vecs.as<double>(), r->lde, static_cast<double*>(dst), ld);
  if (!out_on_device)
    APF_CUDA(cudaMemcpyAsync(out, tmp.p, (size_t)ld * r->e * es, cudaMemcpyDeviceToHost, ctx->stream));
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  APF_CATCH(ctx)
}

apf_status apf_result_stats(const apf_result* r, apf_stats* out) {
  if (!r || !out) return APF_ERR_ARG;
  *out = r->stats;
  return APF_OK;
}

apf_status apf_result_history(const apf_result* r, double* host_out, int32_t cap, int32_t* count) {
  if (!r || !count) return APF_ERR_ARG;
  const int32_t nrec = (int32_t)(r->history.size() / 6);
  *count = nrec;
  if (host_out && cap > 0) memcpy(host_out, r->history.data(), (size_t)std::min(cap, nrec) * 6 * sizeof(double));
  return APF_OK;
}

apf_status apf_result_destroy(apf_result* r) {
  if (!r) return APF_OK;
  apf_ctx* owned = r->owns_ctx ? r->ctx : nullptr;
  if (r->ctx) {
    cudaSetDevice(r->ctx->device);
    cudaStreamSynchronize(r->ctx->stream);
  }
  delete r;
  if (owned) apf_destroy(owned);
  return APF_OK;
}

// ---- the steps one by one ------------------------------------------------------------
apf_status apf_filter_coefficients(double am, double bm, int32_t k, int32_t damping, double m_d,
                                   double* host_out) {
  if (!host_out || k < 0 || !(am > -1.0 && bm < 1.0 && am < bm)) return APF_ERR_ARG;
  if (damping < APF_DAMP_LANCZOS_M || damping > APF_DAMP_NONE) return APF_ERR_ARG;
  const std::vector<double> a = apf::filter_coefficients(am, bm, k, damping, m_d);
  memcpy(host_out, a.data(), a.size() * sizeof(double));
  return APF_OK;
}

apf_status apf_degree_select(const double* ritz, int32_t p, int32_t e, const double* coef, int32_t k,
                             double l1, double l2, double tau_a, int32_t* degree) {
  if (!ritz || !coef || !degree || p < 1 || k < 0) return APF_ERR_ARG;
  *degree = apf::degree_select(ritz, p, e, coef, k, l1, l2, tau_a);
  return APF_OK;
}

apf_status apf_spectrum_bounds(apf_ctx* ctx, const apf_matrix* A, int32_t steps, uint64_t seed,
                               double pad, double* host_out) {
  if (!ctx || !A || !host_out || steps < 1) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  apf::spectrum_bounds(ctx, A, steps, seed, pad, host_out);
  APF_CATCH(ctx)
}

apf_status apf_filter_apply(apf_ctx* ctx, const apf_matrix* A, const double* coef, int32_t degree,
                            double l1, double l2, int32_t precision, const void* X, int64_t ldx,
                            int64_t p, void* Y, int64_t ldy) {
  if (!ctx || !A || !coef || degree < 0 || !X || !Y || p < 1 || ldx < p || ldy < p) return APF_ERR_ARG;
  if (precision != APF_FILTER_F64 && precision != APF_FILTER_F32) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (A->dtype == APF_C128)
    apf::filter_apply_public<double2>(ctx, A, coef, degree, l1, l2, precision, static_cast<const double2*>(X), ldx, p,
                                      static_cast<double2*>(Y), ldy);
  else
    apf::filter_apply_public<double>(ctx, A, coef, degree, l1, l2, precision, static_cast<const double*>(X), ldx, p,
                                     static_cast<double*>(Y), ldy);
  APF_CATCH(ctx)
}

apf_status apf_count_estimate(apf_ctx* ctx, const apf_matrix* A, const double* coef, int32_t degree, double l1,
                              double l2, int32_t precision, int32_t m, uint64_t seed, double* host_out) {
  if (!ctx || !A || !coef || degree < 0 || !host_out || m < 1 || m > 8 * APF_MAX_P) return APF_ERR_ARG;
  if (precision != APF_FILTER_F64 && precision != APF_FILTER_F32) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (A->dtype == APF_C128)
    *host_out = apf::count_estimate_public<double2>(ctx, A, coef, degree, l1, l2, precision, m, seed);
  else
    *host_out = apf::count_estimate_public<double>(ctx, A, coef, degree, l1, l2, precision, m, seed);
  APF_CATCH(ctx)
}

apf_status apf_filter_apply_defect(apf_ctx* ctx, const apf_matrix* A, const double* coef, int32_t degree,
                                   double l1, double l2, const void* V, const void* AV, const double* lam,
                                   int64_t ld, int64_t p, void* Y, int64_t ldy) {
  if (!ctx || !A || !coef || degree < 0 || !V || !AV || !lam || !Y || p < 1 || ld < p || ldy < p)
    return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (A->dtype == APF_C128)
    apf::filter_apply_defect_public<double2>(ctx, A, coef, degree, l1, l2, static_cast<const double2*>(V),
                                             static_cast<const double2*>(AV), lam, ld, p, static_cast<double2*>(Y), ldy);
  else
    apf::filter_apply_defect_public<double>(ctx, A, coef, degree, l1, l2, static_cast<const double*>(V),
                                            static_cast<const double*>(AV), lam, ld, p, static_cast<double*>(Y), ldy);
  APF_CATCH(ctx)
}

apf_status apf_spmm(apf_ctx* ctx, const apf_matrix* A, const void* X, int64_t ldx, int64_t p, void* Y,
                    int64_t ldy) {
  if (!ctx || !A || !X || !Y || p < 1 || ldx < p || ldy < p) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (A->dtype == APF_C128)
    apf::spmm_public<double2>(ctx, A, static_cast<const double2*>(X), ldx, p, static_cast<double2*>(Y), ldy);
  else
    apf::spmm_public<double>(ctx, A, static_cast<const double*>(X), ldx, p, static_cast<double*>(Y), ldy);
  APF_CATCH(ctx)
}

apf_status apf_gram(apf_ctx* ctx, int32_t dtype, int64_t n, int64_t pa, int64_t pb, const void* X,
                    int64_t ldx, const void* Y, int64_t ldy, void* G, int64_t ldg) {
  if (!ctx || !X || !Y || !G || n < 1 || pa < 1 || pb < 1 || ldx < pa || ldy < pb || ldg < pb) return APF_ERR_ARG;
  if (dtype != APF_R64 && dtype != APF_C128) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (dtype == APF_C128)
    apf::gram<double2>(ctx, n, pa, pb, static_cast<const double2*>(X), ldx, static_cast<const double2*>(Y), ldy,
                       static_cast<double2*>(G), ldg, false);
  else
    apf::gram<double>(ctx, n, pa, pb, static_cast<const double*>(X), ldx, static_cast<const double*>(Y), ldy,
                      static_cast<double*>(G), ldg, false);
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  APF_CATCH(ctx)
}

apf_status apf_gram_tc(apf_ctx* ctx, int32_t dtype, int64_t n, int64_t pa, int64_t pb, const void* X,
                       int64_t ldx, const void* Y, int64_t ldy, void* G, int64_t ldg) {
  if (!ctx || !X || !Y || !G || n < 1 || pa < 1 || pb < 1 || ldx < pa || ldy < pb || ldg < pb) return APF_ERR_ARG;
  if (pa > APF_MAX_P || pb > APF_MAX_P) return APF_ERR_ARG;
  if (dtype != APF_R64 && dtype != APF_C128) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (dtype == APF_C128)
    apf::gram_tc<double2>(ctx, n, pa, pb, static_cast<const double2*>(X), ldx, static_cast<const double2*>(Y), ldy,
                          static_cast<double2*>(G), ldg, false);
  else
    apf::gram_tc<double>(ctx, n, pa, pb, static_cast<const double*>(X), ldx, static_cast<const double*>(Y), ldy,
                         static_cast<double*>(G), ldg, false);
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  if (apf::fetch_device_error(ctx) != 0) throw ApfError{APF_ERR_TIMEOUT, "tensor-core Gram"};
  APF_CATCH(ctx)
}

apf_status apf_block_update(apf_ctx* ctx, int32_t dtype, int64_t n, int64_t pa, int64_t pb, const void* X,
                            int64_t ldx, const void* M, int64_t ldm, void* Z, int64_t ldz, double alpha, double beta,
                            int32_t tensor_cores) {
  if (!ctx || !X || !M || !Z || n < 1 || pa < 1 || pb < 1 || pa > APF_MAX_P || pb > APF_MAX_P || ldx < pa ||
      ldm < pb || ldz < pb)
    return APF_ERR_ARG;
  if (dtype != APF_R64 && dtype != APF_C128) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  const double b = beta;
  if (dtype == APF_C128) {
    auto* z = static_cast<double2*>(Z);
    if (tensor_cores)
      apf::gemm_tall_tc<double2>(ctx, n, pa, pb, static_cast<const double2*>(X), ldx, static_cast<const double2*>(M),
                                 ldm, z, ldz, alpha, b, b != 0.0 ? z : nullptr, ldz);
    else
      apf::gemm_tall<double2>(ctx, n, pa, pb, static_cast<const double2*>(X), ldx, static_cast<const double2*>(M),
                              ldm, z, ldz, alpha, b, b != 0.0 ? z : nullptr, ldz, false);
  } else {
    auto* z = static_cast<double*>(Z);
    if (tensor_cores)
      apf::gemm_tall_tc<double>(ctx, n, pa, pb, static_cast<const double*>(X), ldx, static_cast<const double*>(M), ldm,
                                z, ldz, alpha, b, b != 0.0 ? z : nullptr, ldz);
    else
      apf::gemm_tall<double>(ctx, n, pa, pb, static_cast<const double*>(X), ldx, static_cast<const double*>(M), ldm,
                             z, ldz, alpha, b, b != 0.0 ? z : nullptr, ldz, false);
  }
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  if (apf::fetch_device_error(ctx) != 0) throw ApfError{APF_ERR_TIMEOUT, "block update"};
  APF_CATCH(ctx)
}

apf_status apf_cholqr2(apf_ctx* ctx, int32_t dtype, int64_t n, int64_t p, void* X, int64_t ld) {
  if (!ctx || !X || n < 1 || p < 1 || p > n || p > APF_MAX_P || ld < p) return APF_ERR_ARG;
  if (dtype != APF_R64 && dtype != APF_C128) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (dtype == APF_C128) apf::cholqr2_public<double2>(ctx, n, p, static_cast<double2*>(X), ld);
  else apf::cholqr2_public<double>(ctx, n, p, static_cast<double*>(X), ld);
  APF_CATCH(ctx)
}

apf_status apf_eigh_small(apf_ctx* ctx, int32_t dtype, int64_t p, const void* B, int64_t ldb, double* w,
                          void* U, int64_t ldu) {
  if (!ctx || !B || !w || !U || p < 1 || p > APF_MAX_P || ldb < p || ldu < p) return APF_ERR_ARG;
  if (dtype != APF_R64 && dtype != APF_C128) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (dtype == APF_C128)
    apf::eigh_jacobi<double2>(ctx, p, static_cast<const double2*>(B), ldb, w, static_cast<double2*>(U), ldu);
  else
    apf::eigh_jacobi<double>(ctx, p, static_cast<const double*>(B), ldb, w, static_cast<double*>(U), ldu);
  const int derr = apf::fetch_device_error(ctx);
  if (derr == DEV_EIGH_NOCONV) throw ApfError{APF_ERR_EIGH, "eigh"};
  if (derr == DEV_BARRIER_TIMEOUT) throw ApfError{APF_ERR_TIMEOUT, "eigh barrier"};
  if (derr) throw ApfError{APF_ERR_CUDA, "device error"};
  APF_CATCH(ctx)
}

apf_status apf_rayleigh_ritz(apf_ctx* ctx, const apf_matrix* A, const void* Q, int64_t ld, int64_t p,
                             double* w, void* V, int64_t ldv) {
  if (!ctx || !A || !Q || !w || !V || p < 1 || p > APF_MAX_P || ld < p || ldv < p) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (A->dtype == APF_C128)
    apf::rayleigh_ritz_public<double2>(ctx, A, static_cast<const double2*>(Q), ld, p, w, static_cast<double2*>(V), ldv);
  else
    apf::rayleigh_ritz_public<double>(ctx, A, static_cast<const double*>(Q), ld, p, w, static_cast<double*>(V), ldv);
  APF_CATCH(ctx)
}

apf_status apf_residual_norms(apf_ctx* ctx, const apf_matrix* A, const void* V, int64_t ld, int64_t p,
                              const double* w, double* host_out) {
  if (!ctx || !A || !V || !w || !host_out || p < 1 || ld < p) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (A->dtype == APF_C128)
    apf::residual_norms_public<double2>(ctx, A, static_cast<const double2*>(V), ld, p, w, host_out);
  else
    apf::residual_norms_public<double>(ctx, A, static_cast<const double*>(V), ld, p, w, host_out);
  APF_CATCH(ctx)
}

apf_status apf_random_block(apf_ctx* ctx, int32_t dtype, uint64_t seed, uint32_t stream, int64_t n, int64_t p,
                            void* X, int64_t ld) {
  if (!ctx || !X || n < 1 || p < 1 || ld < p) return APF_ERR_ARG;
  if (dtype != APF_R64 && dtype != APF_C128) return APF_ERR_ARG;
  APF_TRY(ctx)
  bind(ctx);
  if (dtype == APF_C128) apf::random_block<double2>(ctx, seed, stream, n, p, static_cast<double2*>(X), ld);
  else apf::random_block<double>(ctx, seed, stream, n, p, static_cast<double*>(X), ld);
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  APF_CATCH(ctx)
}

}  // extern "C"
