// The building blocks of Alg. 4 shared by the single solve, the batched
// spectrum slices (solver.cu) and the serving engine (engine.cu): the
// Clenshaw recurrence over device buffers (Alg. 2), the filter state of one
// solve, Cholesky QR, Rayleigh-Ritz and the residual step, the per-interval
// state of Alg. 4 with its spurious rule, locking and Alg. 3, the count
// estimate of Sec. 3.4 and the set-up of the spectrum bounds.
#pragma once
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <vector>

#include "host_math.h"
#include "solver.h"
#include "spmm_sell_ct.cuh"

namespace apf {

// ---- Alg. 2: the Clenshaw recurrence over device buffers -------------------------------
template <class S>
struct Stepper;

// Counters of the SpMM launches of one filter application.
struct FilterCount {
  int64_t launches = 0;   // kernel launches
  int64_t steps = 0;      // Clenshaw steps (a two-step launch counts 2)
  double bytes = 0.0;     // algorithmic bytes of the launched kernels
  double step_bytes = 0.0;  // algorithmic bytes of the same steps run one per launch
  int kind = -1, G = 0, VPT = 0;  // FP32 step kernel of the first (widest) application
  int64_t graph_replays = 0;      // applications replayed from a captured CUDA graph
  template <class S>
  void note(const Stepper<S>& st) {
    if (kind < 0) { kind = st.kind == 0 ? 3 : st.kind; G = st.G; VPT = st.VPT; }  // internal 0 = CSR
  }
};

static double step_bytes(int64_t n, int64_t nnz, int64_t p, size_t sval, size_t sblk, bool vin,
                         bool y) {
  const double mat = (double)nnz * (double)(sval + 4) + 8.0 * (double)(n + 1);
  const double streams = 2.0 + (vin ? 1.0 : 0.0) + (y ? 1.0 : 0.0);
  return mat + streams * (double)n * (double)p * (double)sblk;
}

// two steps in one pass: A once per step, W and V read once, Y read once,
// both results written (5 block streams; 4 without the first V)
static double pair_bytes(int64_t n, int64_t nnz, int64_t p, size_t sval, size_t sblk, bool vin) {
  const double mat = (double)nnz * (double)(sval + 4) + 8.0 * (double)(n + 1);
  const double streams = 4.0 + (vin ? 1.0 : 0.0);
  return 2.0 * mat + streams * (double)n * (double)p * (double)sblk;
}

// One Clenshaw step of the chosen kernel: CSR or SELL-8 storage of A_hat and
// the (G, VPT) shape picked by the autotuner.
template <class S>
struct Stepper {
  using Real = typename ScalarTraits<S>::Real;
  apf_ctx* ctx = nullptr;
  const apf_matrix* A = nullptr;
  const S* csr_vals = nullptr;   // A_hat values in CSR order
  const S* sell_vals = nullptr;   // A_hat values in natural SELL-8 order (FP32 only), or null
  const S* psell_vals = nullptr;  // A_hat values in permuted SELL-8 order, or null
  size_t seg_bytes = 0;
  int64_t ld = 0;
  // kind 1: SELL, one step per launch; 2: SELL, two steps per launch; 4: SELL,
  // one column tile of G x VPT vectors per CTA (any width); 5: as 4, with the
  // matrix's near rows of W staged in shared memory; 0: CSR
  int kind = 0, G = 0, VPT = 0;
  unsigned* seg_count = nullptr;  // pair-pass counters (kind 2)
  unsigned* pass = nullptr;       // passes made with seg_count
  bool pairs() const { return kind == 2; }
  // bufB = 2 A_hat bufA - va + f1 Y; then bufA = 2 A_hat bufB - bufA + f2 Y
  void pair(S* bufA, S* bufB, const S* va, const S* Y, int64_t ncols, const Real* f1_col, Real f1,
            const Real* f2_col, Real f2) const {
    if constexpr (sizeof(Real) == 4) {
      *pass += 1;
      if (A->perm)  // the banded (permuted) copy
        clenshaw_sell_pair<S, S>(ctx, G, VPT, A->n, A->psell_chunk_ptr, A->psell_col, psell_vals,
                                 A->psell_lmax, A->psell_bw, bufA, bufB, va, Y, ld, ncols, f1_col, f1, f2_col,
                                 f2, seg_count, *pass);
      else
        clenshaw_sell_pair<S, S>(ctx, G, VPT, A->n, A->sell_chunk_ptr, A->sell_col, sell_vals, A->sell_lmax,
                                 A->sell_bw, bufA, bufB, va, Y, ld, ncols, f1_col, f1, f2_col, f2, seg_count,
                                 *pass);
    }
  }
  void operator()(const S* W, const S* Vin, const S* Y, int64_t ncols, const Real* coef_col,
                  Real coef_scalar, Real alpha, S* Out) const {
    if (kind == 4 || kind == 5) {
      if constexpr (sizeof(Real) == 4)
        clenshaw_step_sell_ct<S, S>(ctx, G, VPT, A->n, A->sell_chunk_ptr, A->sell_col, sell_vals, A->sell_lmax, W,
                                    Vin, Y, ld, ncols, coef_col, coef_scalar, alpha, Out,
                                    kind == 5 ? A->sell_halo : 0);
    } else if (kind >= 1) {
      // the two-step form keeps its blocks in the permuted row order: its
      // single steps (the last one or two) must use the permuted copy too
      if constexpr (sizeof(Real) == 4) {
        if (kind == 2 && A->perm)
          clenshaw_step_sell<S, S>(ctx, G, VPT, A->n, A->psell_chunk_ptr, A->psell_col, psell_vals,
                                   A->psell_lmax, W, Vin, Y, ld, ncols, coef_col, coef_scalar, alpha, Out);
        else
          clenshaw_step_sell<S, S>(ctx, G, VPT, A->n, A->sell_chunk_ptr, A->sell_col, sell_vals,
                                   A->sell_lmax, W, Vin, Y, ld, ncols, coef_col, coef_scalar, alpha, Out);
      }
    } else if (G > 0) {
      if constexpr (sizeof(Real) == 4)
        clenshaw_step_shape<S, S>(ctx, G, VPT, A->n, A->rowptr, A->colidx, csr_vals, W, Vin, Y, ld,
                                  ncols, coef_col, coef_scalar, alpha, Out);
    } else {
      clenshaw_step<S, S>(ctx, A->n, A->rowptr, A->colidx, csr_vals, W, Vin, Y, ld, ncols, coef_col,
                          coef_scalar, alpha, Out);
    }
  }
};

constexpr int kNumSellShapes = (int)(sizeof(kSellShapes) / sizeof(kSellShapes[0]));
constexpr int kNumSellCtShapes = (int)(sizeof(kSellCtShapes) / sizeof(kSellCtShapes[0]));

// a column-tiled shape applies when its shared memory fits and the grid's
// tile dimension stays within range
template <class S>
static bool sell_ct_fits(const Stepper<S>& st, int G, int VPT, int nvec, int halo = 0) {
  const int TV = G * VPT;
  return sell_ct_smem_bytes(256 / G, TV, st.A->sell_lmax, sizeof(S), halo) <= 160 * 1024 &&
         256 / G + 2 * halo <= 256 && (nvec + TV - 1) / TV <= 65535 && st.A->n <= INT32_MAX;
}

// idle fraction of the vector slots of the column tiles covering nvec vectors
static double ct_idle(int G, int VPT, int nvec) {
  const int TV = G * VPT, tiles = (nvec + TV - 1) / TV;
  return (double)(tiles * TV - nvec) / (tiles * TV);
}

template <class S>
static bool sell_shape_fits(const Stepper<S>& st, int G, int VPT, int nvec) {
  if (G * VPT < nvec) return false;
  const int R = 256 / G;
  return (size_t)R * st.ld * sizeof(S) * 2 + (size_t)R * st.A->sell_lmax * 12 <= 180 * 1024 &&
         (size_t)R * st.ld * sizeof(S) * 2 + (size_t)R * (st.A->perm ? st.A->psell_lmax : st.A->sell_lmax) * 12 <=
             180 * 1024;
}

// The kernel pinned on the matrix, without timing: kind 2 (two steps per
// pass) falls back to 1 (SELL) and 1 to CSR where they do not apply; the
// pinned (G, VPT) when it covers the width, else the shape with the fewest
// idle vector slots (ties: more vectors per lane).
template <class S>
static void pinned_shape(Stepper<S>& st, int nvec) {
  const apf_matrix* A = st.A;
  int kind = A->pin_kind == 3 ? 0 : A->pin_kind;
  if (kind == 5 && A->sell_halo == 0) kind = 4;
  if (kind == 4 || kind == 5) {
    if (A->sell_ok) {
      const int halo = kind == 5 ? A->sell_halo : 0;
      int bg = 0, bv = 0;
      for (int i = 0; i < kNumSellCtShapes; ++i) {
        const int g = kSellCtShapes[i].G, v = kSellCtShapes[i].VPT;
        if (!sell_ct_fits(st, g, v, nvec, halo)) continue;
        if (g == A->pin_G && v == A->pin_VPT) { bg = g; bv = v; break; }
        if (bg == 0 || ct_idle(g, v, nvec) < ct_idle(bg, bv, nvec) - 1e-12) { bg = g; bv = v; }
      }
      if (bg) { st.kind = kind; st.G = bg; st.VPT = bv; return; }
    }
    kind = 1;
  }
  if (kind >= 1 && !(A->sell_ok && nvec <= 256)) kind = 0;
  if (kind == 2) {
    const int R = 256 / (A->pin_G > 0 ? A->pin_G : 8);
    if (st.seg_count == nullptr || (int64_t)R * 4 >= A->n) kind = 1;
  }
  if (kind == 0) {
    st.kind = 0;
    const int nv = nvec > 256 ? 256 : nvec;
    choose_group(nv, &st.G, &st.VPT);
    static const int csrG[] = {4, 8, 16, 32};
    bool ok = false;
    for (int g : csrG) ok = ok || g == A->pin_G;
    const bool vok = A->pin_VPT >= 1 && A->pin_VPT <= 8 && A->pin_VPT != 7;
    if (ok && vok && A->pin_G * A->pin_VPT >= nv) { st.G = A->pin_G; st.VPT = A->pin_VPT; }
    return;
  }
  int bg = 0, bv = 0;
  for (int i = 0; i < kNumSellShapes; ++i) {
    const int g = kSellShapes[i].G, v = kSellShapes[i].VPT;
    if (!sell_shape_fits(st, g, v, nvec)) continue;
    if (g == A->pin_G && v == A->pin_VPT) { bg = g; bv = v; break; }
    if (bg == 0 || g * v < bg * bv || (g * v == bg * bv && v > bv)) { bg = g; bv = v; }
  }
  if (bg == 0) {  // no SELL shape fits: CSR
    st.kind = 0;
    choose_group(nvec > 256 ? 256 : nvec, &st.G, &st.VPT);
    return;
  }
  if (kind == 2 && (int64_t)(256 / bg) * 4 >= A->n) kind = 1;
  st.kind = kind;
  st.G = bg;
  st.VPT = bv;
}

// Autotuner: time each candidate shape on the live buffers (one warm-up pass
// and four timed steps each, used as the recurrence uses them: Y fixed, the
// output written over V, and each step's output the next step's W) and keep
// the fastest per (element size, ld, width) in the matrix.  All shapes do the same arithmetic in the same order, so the choice
// changes the time, never the result.
template <class S>
static void tune_stepper(Stepper<S>& st, int64_t p, const S* Wb, const S* Yb, S* Ob) {
  using Real = typename ScalarTraits<S>::Real;
  constexpr int E = ScalarTraits<S>::per16;
  st.kind = 0;
  st.G = st.VPT = 0;
  if constexpr (sizeof(Real) != 4) return;
  const int nvec = (int)((p + E - 1) / E);
  apf_matrix* A = const_cast<apf_matrix*>(st.A);
  if (A->pin_kind != 0) {
    pinned_shape(st, nvec);
    return;
  }
  const int64_t key = ((int64_t)sizeof(S) << 48) | ((int64_t)st.ld << 16) | nvec;
  for (auto& kv : A->tune_cache)
    if (kv.first == key) {
      st.kind = kv.second / 10000;
      st.G = (kv.second / 100) % 100;
      st.VPT = kv.second % 100;
      return;
    }
  struct Cand { int kind, G, VPT; };
  std::vector<Cand> cands;
  int g0, v0;
  choose_group(nvec > 256 ? 256 : nvec, &g0, &v0);
  // SELL shapes run in the SELL row order (possibly permuted), CSR in the
  // natural one: a matrix with a SELL copy always uses SELL
  if (!(A->sell_ok && nvec <= 256)) cands.push_back({0, g0, v0});
  if (A->sell_ok && nvec <= 256) {
    const auto& shapes = kSellShapes;
    // shapes with at most 40 % idle vector slots, or the least idle one
    int least = -1;
    for (int i = 0; i < kNumSellShapes; ++i) {
      const int gv = shapes[i].G * shapes[i].VPT;
      if (gv >= nvec && (least < 0 || gv < shapes[least].G * shapes[least].VPT)) least = i;
    }
    for (int i = 0; i < kNumSellShapes; ++i) {
      const int g = shapes[i].G, v = shapes[i].VPT;
      if (g * v < nvec) continue;
      if ((double)(g * v - nvec) / (g * v) > 0.4 && i != least) continue;
      const int R = 256 / g;
      if (!sell_shape_fits(st, g, v, nvec)) continue;
      cands.push_back({1, g, v});
      // two steps per pass when the rows a tile depends on stay within reach of L2
      const int64_t bwp = A->perm ? A->psell_bw : A->sell_bw;
      const double window = (double)(2 * bwp + (PAIR_SEG + 1) * R) * st.ld * sizeof(S) * 3.0;
      if (window <= 64.0 * 1024 * 1024 && (int64_t)R * 4 < A->n) cands.push_back({2, g, v});
    }
  }
  if (A->sell_ok) {
    // column tiles: the shapes with at most 50 % idle slots, or the least idle one
    int least = -1;
    for (int i = 0; i < kNumSellCtShapes; ++i) {
      const int g = kSellCtShapes[i].G, v = kSellCtShapes[i].VPT;
      if (!sell_ct_fits(st, g, v, nvec)) continue;
      if (least < 0 || ct_idle(g, v, nvec) < ct_idle(kSellCtShapes[least].G, kSellCtShapes[least].VPT, nvec))
        least = i;
    }
    for (int i = 0; i < kNumSellCtShapes; ++i) {
      const int g = kSellCtShapes[i].G, v = kSellCtShapes[i].VPT;
      if (!sell_ct_fits(st, g, v, nvec)) continue;
      if (ct_idle(g, v, nvec) > 0.5 && i != least) continue;
      cands.push_back({4, g, v});
      // and with the near rows of W in shared memory, where the matrix has them
      if (A->sell_halo > 0 && sell_ct_fits(st, g, v, nvec, A->sell_halo)) cands.push_back({5, g, v});
    }
  }
  APF_REQUIRE(!cands.empty(), APF_ERR_ARG);
  const bool verbose = getenv("APF_VERBOSE") != nullptr;
  struct EventPair {  // destroyed on every exit, including a failed launch
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  APF_CUDA(cudaEventCreate(&ev.a));
  APF_CUDA(cudaEventCreate(&ev.b));
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  float best = 1e30f;
  Cand pick = cands[0];
  for (const Cand& c : cands) {
    Stepper<S> t = st;
    t.kind = c.kind;
    t.G = c.G;
    t.VPT = c.VPT;
    // time per Clenshaw step: 4 single steps, or 2 two-step passes, on the
    // buffers the way the recurrence uses them: W, Y and V distinct, the
    // output over V (b_j replaces b_{j+2})
    auto run = [&]() {
      if (t.pairs()) {
        APF_CUDA(cudaMemsetAsync(t.seg_count, 0, st.seg_bytes, st.ctx->stream));
        *t.pass = 0;
        t.pair(const_cast<S*>(Wb), Ob, Ob, Yb, p, nullptr, (Real)0.5, nullptr, (Real)0.25);
        t.pair(const_cast<S*>(Wb), Ob, Ob, Yb, p, nullptr, (Real)0.5, nullptr, (Real)0.25);
      } else {
        // each step reads what the one before wrote, as in the recurrence
        S* b[2] = {const_cast<S*>(Wb), Ob};
        for (int r = 0; r < 4; ++r) t(b[r & 1], b[(r + 1) & 1], Yb, p, nullptr, (Real)0.5, (Real)2, b[(r + 1) & 1]);
      }
    };
    if (&c == &cands[0]) run();  // the GPU's clocks settle before the first timing
    run();
    APF_CUDA(cudaEventRecord(e0, st.ctx->stream));
    run();
    APF_CUDA(cudaEventRecord(e1, st.ctx->stream));
    APF_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    APF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (verbose) fprintf(stderr, "apf tune: nvec %d kind %d G %d VPT %d: %.2f us per step\n", nvec, c.kind,
                         c.G, c.VPT, 1e3 * ms / 4.0);
    if (ms < best) { best = ms; pick = c; }
  }
  if (fetch_device_error(st.ctx) != 0) throw ApfError{APF_ERR_TIMEOUT, "filter tuning"};
  st.kind = pick.kind;
  st.G = pick.G;
  st.VPT = pick.VPT;
  if (verbose) fprintf(stderr, "apf tune: nvec %d picked kind %d G %d VPT %d\n", nvec, pick.kind, pick.G, pick.VPT);
  A->tune_cache.push_back({key, pick.kind * 10000 + pick.G * 100 + pick.VPT});
}

// Plain form: returns the buffer (B1 or B2) that holds rho(A_hat) Y.
// a: host coefficients a_0..a_k.  ev0/ev1 bracket the SpMM launches.  With a
// two-step stepper the middle steps run in pairs (b_j and b_{j-1} per pass).
template <class S>
static S* clenshaw_plain(apf_ctx* ctx, const Stepper<S>& step, int64_t n, int64_t nnz, const S* Y,
                         int64_t ld, int64_t p, const double* a, int k, S* B1, S* B2, cudaEvent_t ev0,
                         cudaEvent_t ev1, FilterCount* fc) {
  using Real = typename ScalarTraits<S>::Real;
  if (k == 0) {
    scale_block<S>(ctx, n, p, a[0], Y, ld, B1, ld);
    if (ev0) { APF_CUDA(cudaEventRecord(ev0, ctx->stream)); APF_CUDA(cudaEventRecord(ev1, ctx->stream)); }
    return B1;
  }
  scale_block<S>(ctx, n, p, a[k], Y, ld, B1, ld);  // b_k = a_k Y
  S* P1 = B1;        // b_{j+1}
  S* P2 = nullptr;   // b_{j+2} (zero at the start)
  if (ev0) APF_CUDA(cudaEventRecord(ev0, ctx->stream));
  int j = k - 1;
  while (j >= 0) {
    S* other = P1 == B1 ? B2 : B1;
    if (step.pairs() && j >= 2) {
      // b_j -> other buffer (over b_{j+2}), b_{j-1} -> P1's buffer (over b_{j+1})
      step.pair(P1, other, P2, Y, p, nullptr, (Real)a[j], nullptr, (Real)a[j - 1]);
      fc->launches += 1;
      fc->steps += 2;
      fc->bytes += pair_bytes(n, nnz, p, sizeof(S), sizeof(S), P2 != nullptr);
      fc->step_bytes += step_bytes(n, nnz, p, sizeof(S), sizeof(S), P2 != nullptr, true) +
                        step_bytes(n, nnz, p, sizeof(S), sizeof(S), true, true);
      P2 = other;  // b_j;  P1 now holds b_{j-1}
      j -= 2;
      continue;
    }
    S* out = P2 ? P2 : other;
    const Real alpha = (j == 0) ? (Real)1 : (Real)2;
    step(P1, P2, Y, p, nullptr, (Real)a[j], alpha, out);
    const double b = step_bytes(n, nnz, p, sizeof(S), sizeof(S), P2 != nullptr, true);
    fc->launches += 1;
    fc->steps += 1;
    fc->bytes += b;
    fc->step_bytes += b;
    P2 = P1;
    P1 = out;
    j -= 1;
  }
  if (ev0) APF_CUDA(cudaEventRecord(ev1, ctx->stream));
  return P1;
}

// Defect form: returns the buffer holding D (nullptr when D = 0, i.e. k = 0).
// F: device per-column coefficients, row j at F + j ld (see defect_coefficients).
template <class S>
static S* clenshaw_defect(apf_ctx* ctx, const Stepper<S>& step, int64_t n, int64_t nnz, const S* R,
                          int64_t ld, int64_t p, const float* F, int k, S* B1, S* B2, cudaEvent_t ev0,
                          cudaEvent_t ev1, FilterCount* fc) {
  if (k == 0) {
    if (ev0) { APF_CUDA(cudaEventRecord(ev0, ctx->stream)); APF_CUDA(cudaEventRecord(ev1, ctx->stream)); }
    return nullptr;
  }
  if (k == 1) {
    scale_columns<S>(ctx, n, p, F, R, ld, B1);  // D = beta_1 R_hat
    if (ev0) { APF_CUDA(cudaEventRecord(ev0, ctx->stream)); APF_CUDA(cudaEventRecord(ev1, ctx->stream)); }
    return B1;
  }
  scale_columns<S>(ctx, n, p, F + (int64_t)(k - 1) * ld, R, ld, B1);  // D_{k-1} = 2 a_k R_hat
  S* P1 = B1;
  S* P2 = nullptr;  // D_k = 0
  if (ev0) APF_CUDA(cudaEventRecord(ev0, ctx->stream));
  int j = k - 2;
  while (j >= 0) {
    S* other = P1 == B1 ? B2 : B1;
    if (step.pairs() && j >= 2) {
      step.pair(P1, other, P2, R, p, F + (int64_t)j * ld, 0.0f, F + (int64_t)(j - 1) * ld, 0.0f);
      fc->launches += 1;
      fc->steps += 2;
      fc->bytes += pair_bytes(n, nnz, p, sizeof(S), sizeof(S), P2 != nullptr);
      fc->step_bytes += step_bytes(n, nnz, p, sizeof(S), sizeof(S), P2 != nullptr, true) +
                        step_bytes(n, nnz, p, sizeof(S), sizeof(S), true, true);
      P2 = other;
      j -= 2;
      continue;
    }
    S* out = P2 ? P2 : other;
    const float alpha = (j == 0) ? 1.0f : 2.0f;
    step(P1, P2, R, p, F + (int64_t)j * ld, 0.0f, alpha, out);
    const double b = step_bytes(n, nnz, p, sizeof(S), sizeof(S), P2 != nullptr, true);
    fc->launches += 1;
    fc->steps += 1;
    fc->bytes += b;
    fc->step_bytes += b;
    P2 = P1;
    P1 = out;
    j -= 1;
  }
  if (ev0) APF_CUDA(cudaEventRecord(ev1, ctx->stream));
  return P1;
}

// Batched forms (spectrum slices): per-column coefficient rows F (row j at
// F + j ld) and the active width of every step: columns are ordered by
// decreasing degree, so the columns still identically zero at step j (degree
// below j) are a suffix and are left out.  B1 and B2 must be zero on entry.
template <class S>
static S* clenshaw_plain_cols(apf_ctx* ctx, const Stepper<S>& step, int64_t n, int64_t nnz, const S* Y,
                              int64_t ld, const typename ScalarTraits<S>::Real* F, int K,
                              const std::vector<int64_t>& act, S* B1, S* B2, cudaEvent_t ev0,
                              cudaEvent_t ev1, FilterCount* fc) {
  using Real = typename ScalarTraits<S>::Real;
  scale_columns<S>(ctx, n, act[(size_t)K], F + (int64_t)K * ld, Y, ld, B1);  // b_K
  if (K == 0) {
    if (ev0) { APF_CUDA(cudaEventRecord(ev0, ctx->stream)); APF_CUDA(cudaEventRecord(ev1, ctx->stream)); }
    return B1;
  }
  S* P1 = B1;
  S* P2 = nullptr;
  if (ev0) APF_CUDA(cudaEventRecord(ev0, ctx->stream));
  int j = K - 1;
  while (j >= 0) {
    S* other = P1 == B1 ? B2 : B1;
    if (step.pairs() && j >= 2) {
      const int64_t w = act[(size_t)(j - 1)];
      step.pair(P1, other, P2, Y, w, F + (int64_t)j * ld, (Real)0, F + (int64_t)(j - 1) * ld, (Real)0);
      fc->launches += 1;
      fc->steps += 2;
      fc->bytes += pair_bytes(n, nnz, w, sizeof(S), sizeof(S), P2 != nullptr);
      fc->step_bytes += step_bytes(n, nnz, w, sizeof(S), sizeof(S), P2 != nullptr, true) +
                        step_bytes(n, nnz, w, sizeof(S), sizeof(S), true, true);
      P2 = other;
      j -= 2;
      continue;
    }
    const int64_t w = act[(size_t)j];
    S* out = P2 ? P2 : other;
    const Real alpha = (j == 0) ? (Real)1 : (Real)2;
    step(P1, P2, Y, w, F + (int64_t)j * ld, (Real)0, alpha, out);
    const double b = step_bytes(n, nnz, w, sizeof(S), sizeof(S), P2 != nullptr, true);
    fc->launches += 1;
    fc->steps += 1;
    fc->bytes += b;
    fc->step_bytes += b;
    P2 = P1;
    P1 = out;
    j -= 1;
  }
  if (ev0) APF_CUDA(cudaEventRecord(ev1, ctx->stream));
  return P1;
}

template <class S>
static S* clenshaw_defect_cols(apf_ctx* ctx, const Stepper<S>& step, int64_t n, int64_t nnz, const S* R,
                               int64_t ld, const float* F, int K, const std::vector<int64_t>& act, S* B1,
                               S* B2, cudaEvent_t ev0, cudaEvent_t ev1, FilterCount* fc) {
  // act[j]: columns with degree > j (D_j can be non-zero only there)
  if (K == 0) {
    if (ev0) { APF_CUDA(cudaEventRecord(ev0, ctx->stream)); APF_CUDA(cudaEventRecord(ev1, ctx->stream)); }
    return nullptr;
  }
  if (K == 1) {
    scale_columns<S>(ctx, n, act[0], F, R, ld, B1);
    if (ev0) { APF_CUDA(cudaEventRecord(ev0, ctx->stream)); APF_CUDA(cudaEventRecord(ev1, ctx->stream)); }
    return B1;
  }
  scale_columns<S>(ctx, n, act[(size_t)(K - 1)], F + (int64_t)(K - 1) * ld, R, ld, B1);
  S* P1 = B1;
  S* P2 = nullptr;
  if (ev0) APF_CUDA(cudaEventRecord(ev0, ctx->stream));
  int j = K - 2;
  while (j >= 0) {
    S* other = P1 == B1 ? B2 : B1;
    if (step.pairs() && j >= 2) {
      const int64_t w = act[(size_t)(j - 1)];
      step.pair(P1, other, P2, R, w, F + (int64_t)j * ld, 0.0f, F + (int64_t)(j - 1) * ld, 0.0f);
      fc->launches += 1;
      fc->steps += 2;
      fc->bytes += pair_bytes(n, nnz, w, sizeof(S), sizeof(S), P2 != nullptr);
      fc->step_bytes += step_bytes(n, nnz, w, sizeof(S), sizeof(S), P2 != nullptr, true) +
                        step_bytes(n, nnz, w, sizeof(S), sizeof(S), true, true);
      P2 = other;
      j -= 2;
      continue;
    }
    const int64_t w = act[(size_t)j];
    S* out = P2 ? P2 : other;
    const float alpha = (j == 0) ? 1.0f : 2.0f;
    step(P1, P2, R, w, F + (int64_t)j * ld, 0.0f, alpha, out);
    const double b = step_bytes(n, nnz, w, sizeof(S), sizeof(S), P2 != nullptr, true);
    fc->launches += 1;
    fc->steps += 1;
    fc->bytes += b;
    fc->step_bytes += b;
    P2 = P1;
    P1 = out;
    j -= 1;
  }
  if (ev0) APF_CUDA(cudaEventRecord(ev1, ctx->stream));
  return P1;
}

// Filter state of one solve: scaled copies of A and the recurrence buffers.
// With a SELL copy of A the FP32 recurrence runs in the SELL row order (the
// reverse Cuthill-McKee order when the matrix was permuted): rows are mapped on
// the way in (perm: new -> old) and on the way out (iperm: old -> new).
template <class T>
struct FilterState {
  using TL = typename LowOf<T>::type;
  apf_ctx* ctx = nullptr;
  const apf_matrix* A = nullptr;
  int64_t n = 0, ld = 0;
  double l1 = 0, l2 = 0;
  DBuf Ahat64, Ahat32, Asell32, Apsell32;  // l1 A + l2 I: FP64 / FP32 CSR, SELL-8, permuted SELL-8
  DBuf B1, B2, Y32;              // recurrence buffers
  DBuf coef_dev;                 // a_j on the device (defect form)
  DBuf F, rho;                   // defect coefficients
  DBuf segs;                     // two-step pass counters
  unsigned pass = 0;
  // CUDA graphs of the recurrence: one per (form, degree, width, input,
  // kernel), captured the second time that application recurs and replayed
  // afterwards.  The plain form's coefficients are the same for a given degree
  // and the defect form's are device arrays, so a replay does the same work
  // as the launches it replaces.  Not used with the two-step kernel (its
  // pass counters change from launch to launch).
  struct GraphEntry {
    int form = 0, k = 0, kind = 0, G = 0, VPT = 0, seen = 0;
    int64_t p = 0;
    uint64_t sig = 0;  // batched filters: per-column degrees and coefficient table
    const void* in = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* out = nullptr;
    FilterCount fc;
    int64_t launches = 0;
  };
  std::vector<GraphEntry> graphs;
  bool graphs_on = false;
  DBuf Fcols;  // coefficient table of a batched filter ((K + 1) x ld), kept so graphs can replay on it
  std::vector<double> a;         // host a_j
  int precision = APF_FILTER_F64;
  int kmax = 0;

  void init(apf_ctx* c, const apf_matrix* M, int64_t width_ld, double L1, double L2,
            const std::vector<double>& coef, int prec) {
    ctx = c;
    A = M;
    n = M->n;
    ld = width_ld;
    l1 = L1;
    l2 = L2;
    a = coef;
    precision = prec;
    kmax = (int)coef.size() - 1;
    const T* vals = static_cast<const T*>(A->vals);
    if (prec == APF_FILTER_F64) {
      Ahat64.alloc((size_t)A->nnz * sizeof(T), ctx->stream, false);
      scale_shift_matrix<T, T>(ctx, n, A->rowptr, A->colidx, vals, l1, l2, Ahat64.as<T>());
      B1.alloc((size_t)n * ld * sizeof(T), ctx->stream, true);
      B2.alloc((size_t)n * ld * sizeof(T), ctx->stream, true);
    } else {
      Ahat32.alloc((size_t)A->nnz * sizeof(TL), ctx->stream, false);
      scale_shift_matrix<T, TL>(ctx, n, A->rowptr, A->colidx, vals, l1, l2, Ahat32.as<TL>());
      if (A->sell_ok) {
        Asell32.alloc((size_t)A->sell_slots * sizeof(TL), ctx->stream, false);
        sell_gather_values<TL>(ctx, A->sell_slots, A->sell_src, Ahat32.as<TL>(), Asell32.as<TL>());
        if (A->perm) {
          Apsell32.alloc((size_t)A->psell_slots * sizeof(TL), ctx->stream, false);
          sell_gather_values<TL>(ctx, A->psell_slots, A->psell_src, Ahat32.as<TL>(), Apsell32.as<TL>());
        }
        segs.alloc(seg_bytes(), ctx->stream, true);
      }
      B1.alloc((size_t)n * ld * sizeof(TL), ctx->stream, true);
      B2.alloc((size_t)n * ld * sizeof(TL), ctx->stream, true);
      Y32.alloc((size_t)n * ld * sizeof(TL), ctx->stream, true);
      if (!coef.empty()) {  // a batched filter brings its own coefficients
        coef_dev.alloc(coef.size() * sizeof(double), ctx->stream, false);
        APF_CUDA(cudaMemcpyAsync(coef_dev.p, coef.data(), coef.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, ctx->stream));
        F.alloc((size_t)(kmax + 1) * ld * sizeof(float), ctx->stream, true);
      }
      rho.alloc((size_t)ld * sizeof(double), ctx->stream, true);
    }
  }

  ~FilterState() {
    for (auto& g : graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
  }

  // Run body(ev0, ev1, fc) (the launches of one recurrence; returns its output
  // buffer) directly or through a cached graph.
  template <class S, class Body>
  S* run_recurrence(int form, int k, int64_t p, const void* in, const Stepper<S>& st, cudaEvent_t ev0,
                    cudaEvent_t ev1, FilterCount* fc, Body&& body, uint64_t sig = 0) {
    if (!graphs_on || st.pairs()) return body(ev0, ev1, fc);
    GraphEntry* g = nullptr;
    for (auto& e : graphs)
      if (e.form == form && e.k == k && e.p == p && e.in == in && e.kind == st.kind && e.G == st.G &&
          e.VPT == st.VPT && e.sig == sig)
        g = &e;
    if (g == nullptr) {
      GraphEntry e;
      e.form = form; e.k = k; e.p = p; e.in = in; e.kind = st.kind; e.G = st.G; e.VPT = st.VPT; e.sig = sig;
      graphs.push_back(e);
      g = &graphs.back();
    }
    if (g->exec == nullptr && ++g->seen < 2) return body(ev0, ev1, fc);  // first time: run it directly
    if (g->exec == nullptr) {
      if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();  // e.g. the legacy default stream: no capture, no graphs
        graphs_on = false;
        return body(ev0, ev1, fc);
      }
      FilterCount local;
      const int64_t l0 = ctx->launches;
      S* out = nullptr;
      try {
        out = body(nullptr, nullptr, &local);
      } catch (...) {
        cudaGraph_t gr = nullptr;
        cudaStreamEndCapture(ctx->stream, &gr);
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        throw;
      }
      cudaGraph_t gr = nullptr;
      APF_CUDA(cudaStreamEndCapture(ctx->stream, &gr));
      const cudaError_t ie = cudaGraphInstantiate(&g->exec, gr, 0);
      cudaGraphDestroy(gr);
      APF_CUDA(ie);
      g->out = out;
      g->fc = local;
      g->launches = ctx->launches - l0;
      ctx->launches = l0;  // counted again below, at the replay
    }
    if (ev0) APF_CUDA(cudaEventRecord(ev0, ctx->stream));
    APF_CUDA(cudaGraphLaunch(g->exec, ctx->stream));
    if (ev1) APF_CUDA(cudaEventRecord(ev1, ctx->stream));
    ctx->launches += g->launches;
    fc->graph_replays += 1;
    fc->launches += g->fc.launches;
    fc->steps += g->fc.steps;
    fc->bytes += g->fc.bytes;
    fc->step_bytes += g->fc.step_bytes;
    return static_cast<S*>(g->out);
  }

  // counters for the smallest tile (8 rows): ceil(n / 8 / 32) segments
  size_t seg_bytes() const { return (size_t)((n + 8 * PAIR_SEG - 1) / (8 * PAIR_SEG) + 1) * sizeof(unsigned); }

  // row maps of the FP32 recurrence: the two-step form of a permuted matrix
  // runs in the permuted order (null: natural order)
  const int32_t* rows_in(const Stepper<TL>& st) const { return st.pairs() ? A->perm : nullptr; }
  const int32_t* rows_out(const Stepper<TL>& st) const { return st.pairs() ? A->iperm : nullptr; }

  Stepper<T> stepper64() const {
    Stepper<T> s;
    s.ctx = ctx;
    s.A = A;
    s.csr_vals = Ahat64.as<T>();
    s.ld = ld;
    return s;
  }

  // the tuned FP32 stepper for width p (tuning overwrites B1 and B2: call before use)
  Stepper<TL> stepper32(int64_t p) {
    Stepper<TL> s;
    s.ctx = ctx;
    s.A = A;
    s.csr_vals = Ahat32.as<TL>();
    s.sell_vals = A->sell_ok ? Asell32.as<TL>() : nullptr;
    s.psell_vals = A->perm ? Apsell32.as<TL>() : nullptr;
    s.ld = ld;
    s.seg_count = A->sell_ok ? segs.as<unsigned>() : nullptr;
    s.seg_bytes = A->sell_ok ? seg_bytes() : 0;
    s.pass = &pass;
    tune_stepper<TL>(s, p, B1.as<TL>(), Y32.as<TL>(), B2.as<TL>());
    if (s.pairs()) {  // fresh counters for this application's passes
      APF_CUDA(cudaMemsetAsync(segs.p, 0, seg_bytes(), ctx->stream));
      pass = 0;
    }
    return s;
  }

  // X = rho(A_hat) V with degree k; V, X: n x p (ld).  For the defect form AV
  // and lam (device) hold A V and the Ritz values of V; pass nullptr to use the
  // plain FP32 recurrence instead.
  void apply(int k, const T* V, const T* AV, const double* lam, int64_t p, T* X, cudaEvent_t ev0,
             cudaEvent_t ev1, FilterCount* fc) {
    APF_REQUIRE(k <= kmax, APF_ERR_ARG);
    const int64_t nnz = A->nnz;
    if (precision == APF_FILTER_F64) {
      const Stepper<T> s64 = stepper64();
      T* out = run_recurrence<T>(0, k, p, V, s64, ev0, ev1, fc, [&](cudaEvent_t e0, cudaEvent_t e1, FilterCount* f) {
        return clenshaw_plain<T>(ctx, s64, n, nnz, V, ld, p, a.data(), k, B1.as<T>(), B2.as<T>(), e0, e1, f);
      });
      copy_block<T>(ctx, n, p, out, ld, X, ld);
      return;
    }
    const Stepper<TL> st = stepper32(p);
    if (fc) fc->note(st);
    if (precision == APF_FILTER_F32_DEFECT && AV != nullptr && lam != nullptr) {
      // R_hat = l1 (A V - V diag(lam)) in FP32, in the recurrence's row order;
      // the norms are not needed here
      DBuf scratch((size_t)p * sizeof(double), ctx->stream, false);
      residual_norms<T>(ctx, n, p, AV, V, ld, lam, scratch.as<double>(), Y32.as<TL>(), l1, rows_out(st));
      defect_coefficients(ctx, p, ld, k, coef_dev.as<double>(), lam, l1, l2, F.as<float>(), rho.as<double>());
      TL* D = run_recurrence<TL>(1, k, p, Y32.p, st, ev0, ev1, fc, [&](cudaEvent_t e0, cudaEvent_t e1, FilterCount* f) {
        return clenshaw_defect<TL>(ctx, st, n, nnz, Y32.as<TL>(), ld, p, F.as<float>(), k, B1.as<TL>(),
                                   B2.as<TL>(), e0, e1, f);
      });
      defect_combine<T>(ctx, n, p, V, ld, rho.as<double>(), D, ld, X, ld, rows_out(st));
      return;
    }
    cast_block_rows<T, TL>(ctx, n, p, V, ld, Y32.as<TL>(), ld, rows_in(st));
    TL* out = run_recurrence<TL>(2, k, p, Y32.p, st, ev0, ev1, fc, [&](cudaEvent_t e0, cudaEvent_t e1, FilterCount* f) {
      return clenshaw_plain<TL>(ctx, st, n, nnz, Y32.as<TL>(), ld, p, a.data(), k, B1.as<TL>(), B2.as<TL>(), e0,
                                e1, f);
    });
    cast_block_rows<TL, T>(ctx, n, p, out, ld, X, ld, rows_out(st));
  }

  // Batched filter (spectrum slices): column c of V (n x p) is filtered with
  // its own coefficients coef_dev + coff[c] (device) of degree kc[c] (host,
  // non-increasing in c).  Same forms and precisions as apply().
  void apply_cols(const std::vector<int32_t>& kc, const std::vector<int64_t>& coff, const double* coef_dev,
                  const T* V, const T* AV, const double* lam, int64_t p, T* X, cudaEvent_t ev0, cudaEvent_t ev1,
                  FilterCount* fc) {
    APF_REQUIRE((int64_t)kc.size() == p && (int64_t)coff.size() == p && p >= 1, APF_ERR_ARG);
    const int K = kc[0];
    for (int64_t c = 1; c < p; ++c) APF_REQUIRE(kc[(size_t)c] <= kc[(size_t)c - 1], APF_ERR_ARG);
    const int64_t nnz = A->nnz;
    std::vector<int64_t> act_plain((size_t)K + 1, 0), act_def((size_t)K + 1, 0);
    for (int j = 0; j <= K; ++j) {
      int64_t wp = 0, wd = 0;
      while (wp < p && kc[(size_t)wp] >= j) ++wp;
      while (wd < p && kc[(size_t)wd] > j) ++wd;
      act_plain[(size_t)j] = wp;
      act_def[(size_t)j] = wd;
    }
    DBuf kcd((size_t)p * sizeof(int32_t), ctx->stream, false), cod((size_t)p * sizeof(int64_t), ctx->stream, false);
    APF_CUDA(cudaMemcpyAsync(kcd.p, kc.data(), (size_t)p * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    APF_CUDA(cudaMemcpyAsync(cod.p, coff.data(), (size_t)p * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
    // the coefficient table stays in one buffer (grown when needed) and the
    // recurrence's launches depend only on the per-column degrees and that
    // buffer, so a recurring application replays as a CUDA graph
    const size_t fbytes = (size_t)(K + 1) * ld * (precision == APF_FILTER_F64 ? sizeof(double) : sizeof(float));
    if (Fcols.bytes < fbytes) Fcols.alloc(fbytes + fbytes / 4, ctx->stream, false);
    uint64_t sig = 1469598103934665603ull;  // FNV-1a over the degrees and the table's address
    auto mix = [&](uint64_t v) {
      for (int b = 0; b < 8; ++b) { sig ^= (v >> (8 * b)) & 0xFF; sig *= 1099511628211ull; }
    };
    for (int32_t kk : kc) mix((uint64_t)(uint32_t)kk);
    mix((uint64_t)(uintptr_t)Fcols.p);
    if (precision == APF_FILTER_F64) {
      APF_CUDA(cudaMemsetAsync(B1.p, 0, B1.bytes, ctx->stream));
      APF_CUDA(cudaMemsetAsync(B2.p, 0, B2.bytes, ctx->stream));
      coef_columns<double>(ctx, p, ld, K, coef_dev, cod.as<int64_t>(), kcd.as<int32_t>(), nullptr, l1, l2,
                           Fcols.as<double>(), nullptr);
      const Stepper<T> s64 = stepper64();
      T* out = run_recurrence<T>(
          3, K, p, V, s64, ev0, ev1, fc,
          [&](cudaEvent_t e0, cudaEvent_t e1, FilterCount* f) {
            return clenshaw_plain_cols<T>(ctx, s64, n, nnz, V, ld, Fcols.as<double>(), K, act_plain, B1.as<T>(),
                                          B2.as<T>(), e0, e1, f);
          },
          sig);
      copy_block<T>(ctx, n, p, out, ld, X, ld);
      return;
    }
    const Stepper<TL> st = stepper32(p);
    if (fc) fc->note(st);
    APF_CUDA(cudaMemsetAsync(B1.p, 0, B1.bytes, ctx->stream));
    APF_CUDA(cudaMemsetAsync(B2.p, 0, B2.bytes, ctx->stream));
    float* Ff = Fcols.as<float>();
    if (precision == APF_FILTER_F32_DEFECT && AV != nullptr && lam != nullptr) {
      DBuf scratch((size_t)p * sizeof(double), ctx->stream, false);
      residual_norms<T>(ctx, n, p, AV, V, ld, lam, scratch.as<double>(), Y32.as<TL>(), l1, rows_out(st));
      coef_columns<float>(ctx, p, ld, K, coef_dev, cod.as<int64_t>(), kcd.as<int32_t>(), lam, l1, l2, Ff,
                          rho.as<double>());
      TL* D = run_recurrence<TL>(
          4, K, p, Y32.p, st, ev0, ev1, fc,
          [&](cudaEvent_t e0, cudaEvent_t e1, FilterCount* f) {
            return clenshaw_defect_cols<TL>(ctx, st, n, nnz, Y32.as<TL>(), ld, Ff, K, act_def, B1.as<TL>(),
                                            B2.as<TL>(), e0, e1, f);
          },
          sig);
      defect_combine<T>(ctx, n, p, V, ld, rho.as<double>(), D, ld, X, ld, rows_out(st));
      return;
    }
    cast_block_rows<T, TL>(ctx, n, p, V, ld, Y32.as<TL>(), ld, rows_in(st));
    coef_columns<float>(ctx, p, ld, K, coef_dev, cod.as<int64_t>(), kcd.as<int32_t>(), nullptr, l1, l2, Ff,
                        nullptr);
    TL* out = run_recurrence<TL>(
        5, K, p, Y32.p, st, ev0, ev1, fc,
        [&](cudaEvent_t e0, cudaEvent_t e1, FilterCount* f) {
          return clenshaw_plain_cols<TL>(ctx, st, n, nnz, Y32.as<TL>(), ld, Ff, K, act_plain, B1.as<TL>(),
                                         B2.as<TL>(), e0, e1, f);
        },
        sig);
    cast_block_rows<TL, T>(ctx, n, p, out, ld, X, ld, rows_out(st));
  }
};

// ---- Alg. 4, orthogonalisation: Cholesky QR ------------------------------------------------------
template <class T>
static bool cholesky_checked(apf_ctx* ctx, int64_t p, T* G, int64_t ldg, double shift) {
  cholesky_upper<T>(ctx, p, G, ldg, shift);
  const int e = fetch_device_error(ctx);
  if (e == DEV_CHOL_PIVOT) return false;
  if (e != 0) throw ApfError{APF_ERR_CUDA, "device error in Cholesky"};
  return true;
}

// Small p x p workspace of the orthogonalisation and Rayleigh-Ritz steps.
template <class T>
struct SmallWork {
  DBuf buf;
  int64_t p = 0;
  T *G, *Ri, *G3, *T1, *B, *U, *M, *C;
  double* w;
  void init(int64_t pmax, cudaStream_t s) {
    p = pmax;
    const size_t mat = (size_t)pmax * pmax;
    buf.alloc(mat * 8 * sizeof(T) + (size_t)pmax * sizeof(double) + 256, s, true);
    T* b = buf.as<T>();
    G = b;
    Ri = b + mat;
    G3 = b + 2 * mat;
    T1 = b + 3 * mat;
    B = b + 4 * mat;
    U = b + 5 * mat;
    M = b + 6 * mat;
    C = b + 7 * mat;
    w = reinterpret_cast<double*>(b + 8 * mat);
  }
};

// The Gram product on the FP64 cores or on the tensor cores (bf16 slicing).
template <class T>
static void gram_on(apf_ctx* ctx, bool tc, int64_t n, int64_t pa, int64_t pb, const T* X, int64_t ldx, const T* Y,
                    int64_t ldy, T* G, int64_t ldg, bool hermitian) {
  if (tc) gram_tc<T>(ctx, n, pa, pb, X, ldx, Y, ldy, G, ldg, hermitian);
  else gram<T>(ctx, n, pa, pb, X, ldx, Y, ldy, G, ldg, hermitian);
}

// Z = beta Z0 + alpha X M on the FP64 cores or on the tensor cores.
template <class T>
static void gemm_on(apf_ctx* ctx, bool tc, int64_t n, int64_t pa, int64_t pb, const T* X, int64_t ldx, const T* M,
                    int64_t ldm, T* Z, int64_t ldz, double alpha, double beta, const T* Z0, int64_t ldz0,
                    bool upper) {
  if (tc) gemm_tall_tc<T>(ctx, n, pa, pb, X, ldx, M, ldm, Z, ldz, alpha, beta, Z0, ldz0);
  else gemm_tall<T>(ctx, n, pa, pb, X, ldx, M, ldm, Z, ldz, alpha, beta, Z0, ldz0, upper);
}

// One Cholesky QR pass Xout = X R^{-1}, R from G = X^H X (+ shift I).
template <class T>
static bool cholqr_pass(apf_ctx* ctx, int64_t n, int64_t p, const T* X, int64_t ld, T* Xout,
                        SmallWork<T>& sw, bool shifted, bool tc = false) {
  gram_on<T>(ctx, tc, n, p, p, X, ld, X, ld, sw.G, p, true);
  double shift = 0.0;
  if (shifted) {
    // shifted Cholesky QR (Fukaya et al. 2020): s = 11 (n p + p (p + 1)) u ||X||_F^2
    std::vector<T> hG((size_t)p * p);
    APF_CUDA(cudaMemcpyAsync(hG.data(), sw.G, hG.size() * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
    APF_CUDA(cudaStreamSynchronize(ctx->stream));
    double tr = 0.0;
    for (int64_t i = 0; i < p; ++i) tr += real_(hG[(size_t)(i * p + i)]);
    shift = 11.0 * ((double)n * p + (double)p * (p + 1)) * 1.1102230246251565e-16 * tr;
  }
  if (!cholesky_checked<T>(ctx, p, sw.G, p, shift)) return false;
  tri_inv_upper<T>(ctx, p, sw.G, p, sw.Ri, p);
  gemm_on<T>(ctx, tc, n, p, p, X, ld, sw.Ri, p, Xout, ld, 1.0, 0.0, nullptr, ld, true);
  return true;
}

// CholQR2 of X into X (X1 is scratch of the same shape).  Shifted CholQR3 when
// the first factorisation breaks down.
template <class T>
static void cholqr2_inplace(apf_ctx* ctx, int64_t n, int64_t p, T* X, T* X1, int64_t ld,
                            SmallWork<T>& sw) {
  if (!cholqr_pass<T>(ctx, n, p, X, ld, X1, sw, false)) {
    if (!cholqr_pass<T>(ctx, n, p, X, ld, X1, sw, true)) throw ApfError{APF_ERR_CHOL, "shifted CholQR"};
    if (!cholqr_pass<T>(ctx, n, p, X1, ld, X, sw, false)) throw ApfError{APF_ERR_CHOL, "CholQR3"};
    copy_block<T>(ctx, n, p, X, ld, X1, ld);
  }
  if (!cholqr_pass<T>(ctx, n, p, X1, ld, X, sw, false)) throw ApfError{APF_ERR_CHOL, "CholQR2"};
}

template <class T>
static void spmm_plain(apf_ctx* ctx, const apf_matrix* A, const T* X, int64_t ld, int64_t p, T* Y) {
  clenshaw_step<T, T>(ctx, A->n, A->rowptr, A->colidx, static_cast<const T*>(A->vals), X, nullptr,
                      nullptr, ld, p, nullptr, 0.0, 1.0, Y);
}

// Alg. 4 orthogonalisation, Rayleigh-Ritz and residual steps: X (filtered, n x p, destroyed) ->
// Vh = Ritz vectors, AVh = A Vh, w = Ritz values (ascending), res = residual norms.
// CholQR2's second pass is merged with Rayleigh-Ritz:
//   X1 = X R1^{-1};  G2 = X1^H X1 = R2^H R2;  G3 = X1^H (A X1);
//   B = R2^{-H} G3 R2^{-1} = Q^H A Q for Q = X1 R2^{-1};  B = U diag(w) U^H;
//   Vh = Q U = X1 (R2^{-1} U).
template <class T>
static void orth_rr(apf_ctx* ctx, const apf_matrix* A, int64_t p, int64_t ld, T* X, T* X1,
                    const T* Vlock, int64_t nlock, int64_t ldl, SmallWork<T>& sw, T* Vh, T* AVh,
                    double* w, double* res, bool tc) {
  const int64_t n = A->n;
  for (int pass = 0; pass < 2 && nlock > 0; ++pass) {
    gram_on<T>(ctx, tc, n, nlock, p, Vlock, ldl, X, ld, sw.C, p, false);
    gemm_on<T>(ctx, tc, n, nlock, p, Vlock, ldl, sw.C, p, X, ld, -1.0, 1.0, X, ld, false);
  }
  if (!cholqr_pass<T>(ctx, n, p, X, ld, X1, sw, false, tc)) {
    if (!cholqr_pass<T>(ctx, n, p, X, ld, X1, sw, true, tc)) throw ApfError{APF_ERR_CHOL, "shifted CholQR"};
    if (!cholqr_pass<T>(ctx, n, p, X1, ld, X, sw, false, tc)) throw ApfError{APF_ERR_CHOL, "CholQR3"};
    copy_block<T>(ctx, n, p, X, ld, X1, ld);
  }
  T* AX = X;  // X is dead: reuse it for A X1
  spmm_plain<T>(ctx, A, X1, ld, p, AX);
  gram_on<T>(ctx, tc, n, p, p, X1, ld, X1, ld, sw.G, p, true);
  gram_on<T>(ctx, tc, n, p, p, X1, ld, AX, ld, sw.G3, p, true);  // X1^H A X1 is Hermitian
  if (!cholesky_checked<T>(ctx, p, sw.G, p, 0.0)) throw ApfError{APF_ERR_CHOL, "CholQR2 second pass"};
  tri_inv_upper<T>(ctx, p, sw.G, p, sw.Ri, p);
  small_gemm<T>(ctx, p, p, p, 'N', sw.G3, p, 'N', sw.Ri, p, sw.T1, p, 1.0, 0.0);
  small_gemm<T>(ctx, p, p, p, 'H', sw.Ri, p, 'N', sw.T1, p, sw.B, p, 1.0, 0.0);
  symmetrize<T>(ctx, p, sw.B, p);
  eigh_jacobi<T>(ctx, p, sw.B, p, w, sw.U, p);
  small_gemm<T>(ctx, p, p, p, 'N', sw.Ri, p, 'N', sw.U, p, sw.M, p, 1.0, 0.0);
  gemm_on<T>(ctx, tc, n, p, p, X1, ld, sw.M, p, Vh, ld, 1.0, 0.0, nullptr, ld, false);
  spmm_plain<T>(ctx, A, Vh, ld, p, AVh);
  residual_norms<T>(ctx, n, p, AVh, Vh, ld, w, res, nullptr, 0.0);
}

// ---- Alg. 4 for one interval ---------------------------------------------------------------
// The subspace state of one interval [a, b]: its filter (degrees, coefficients),
// the active block and the locked pairs.  A single solve runs one; a batched
// solve runs one per spectrum slice and filters their blocks together.
template <class T>
struct IntervalState {
  double a = 0, b = 0;
  int64_t p = 0, ld = 0;
  int k1 = 0, kmax = 0;
  std::vector<double> coef;  // a_j, j = 0..kmax
  DBuf Vh, AVh, X, X1, Vlock, wv, resv, idxd;
  double* w = nullptr;   // Ritz values (device), then a gather scratch at w + ld
  double* res = nullptr;  // residual norms (device)
  int64_t pa = 0, nlock = 0;
  int ki = 0, n_check_prev = 0;
  bool have_ritz = false;  // Vh holds Ritz vectors with values in w and A Vh in AVh
  bool done = false;       // every in-interval pair locked
  std::vector<double> lam_lock, hw, hr;
  std::vector<double> rec;  // history row of the last iteration

  // set-up (Alg. 4): the map of [a, b], the degrees k^(1) and k, the coefficients
  void setup_filter(const apf_params* prm, double a_, double b_, double l1, double l2) {
    a = a_;
    b = b_;
    APF_REQUIRE(a < b, APF_ERR_ARG);
    const double am = l1 * a + l2, bm = l1 * b + l2;
    APF_REQUIRE(am > -1.0 && bm < 1.0 && am < bm, APF_ERR_ARG);
    if (prm->k_fixed > 0) {
      k1 = kmax = prm->k_fixed;
    } else {
      k1 = initial_degree(am, bm, prm->C);
      kmax = (int)ceil(prm->k_ratio * k1);
    }
    APF_REQUIRE(k1 >= 0 && kmax <= prm->max_degree_cap, APF_ERR_ARG);
    coef = filter_coefficients(am, bm, kmax, prm->damping, prm->m_d);
  }

  // set-up (Alg. 4): buffers for subspace size p and the orthonormal initial block
  void init_block(apf_ctx* ctx, const apf_matrix* A, const apf_params* prm, int64_t p_, uint32_t stream,
                  SmallWork<T>& sw) {
    p = p_;
    const int64_t n = A->n;
    APF_REQUIRE(p >= 1 && p <= n && p <= APF_MAX_P, APF_ERR_ARG);
    ld = block_ld(p);
    const size_t blk = (size_t)n * ld * sizeof(T);
    Vh.alloc(blk, ctx->stream, true);
    AVh.alloc(blk, ctx->stream, true);
    X.alloc(blk, ctx->stream, true);
    X1.alloc(blk, ctx->stream, true);
    Vlock.alloc(blk, ctx->stream, true);
    wv.alloc(sizeof(double) * (size_t)(2 * ld + 8), ctx->stream, true);
    resv.alloc(sizeof(double) * (size_t)(ld + 8), ctx->stream, true);
    idxd.alloc(sizeof(int32_t) * (size_t)(2 * ld + 8), ctx->stream, false);
    w = wv.as<double>();
    res = resv.as<double>();
    hw.assign((size_t)p, 0.0);
    hr.assign((size_t)p, 0.0);
    pa = p;
    ki = k1;
    if (prm->init_block) {
      APF_CUDA(cudaMemcpy2DAsync(Vh.p, ld * sizeof(T), prm->init_block, p * sizeof(T), p * sizeof(T), n,
                                 prm->init_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 ctx->stream));
    } else {
      random_block<T>(ctx, prm->seed, stream, n, p, Vh.as<T>(), ld);
    }
    cholqr2_inplace<T>(ctx, n, p, Vh.as<T>(), X1.as<T>(), ld, sw);
  }

  // after the filter wrote X: orthogonalisation against the locked vectors,
  // Rayleigh-Ritz and residual norms, and the copies of w and res to the host
  // (complete after the next synchronisation)
  void orth(apf_ctx* ctx, const apf_matrix* A, SmallWork<T>& sw, bool tc) {
    orth_rr<T>(ctx, A, pa, ld, X.as<T>(), X1.as<T>(), Vlock.as<T>(), nlock, ld, sw, Vh.as<T>(), AVh.as<T>(),
               w, res, tc);
    APF_CUDA(cudaMemcpyAsync(hw.data(), w, (size_t)pa * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    APF_CUDA(cudaMemcpyAsync(hr.data(), res, (size_t)pa * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  }

  // on the host values of orth(): in-interval count, next degree (Alg. 3),
  // spurious-value rule (Eq. (tau_s)), locking and compaction of the block
  void check(apf_ctx* ctx, const apf_matrix* A, const apf_params* prm, double l1, double l2, double normA) {
    const int64_t n = A->n;
    have_ritz = true;
    std::vector<int> I;
    for (int c = 0; c < pa; ++c)
      if (hw[(size_t)c] >= a && hw[(size_t)c] <= b) I.push_back(c);
    const int e = (int)I.size();
    double maxres = 0.0;
    for (int c : I) maxres = std::max(maxres, hr[(size_t)c] / normA);
    rec = {(double)ki, (double)pa, (double)e, 0.0, (double)nlock, maxres};
    if (e == 0) return;  // no Ritz value inside: same degree again
    const int k_next =
        prm->k_fixed > 0 ? ki : degree_select(hw.data(), (int)pa, e, coef.data(), kmax, l1, l2, prm->tau_a);
    if (prm->spurious_rule) {
      double tau_s = 1e300;
      for (int c : I) tau_s = std::min(tau_s, std::min(fabs(hw[(size_t)c] - a), fabs(hw[(size_t)c] - b)));
      std::vector<int> Cs;
      for (int c : I)
        if (hr[(size_t)c] < tau_s) Cs.push_back(c);
      const int n_check = (int)Cs.size() + (int)nlock;
      if (n_check > 0 && n_check == n_check_prev) I = Cs;
      n_check_prev = n_check;
    }
    // lock converged pairs (implicit deflation, Sec. 3.3.3)
    std::vector<int> L, keep;
    std::vector<char> inL((size_t)pa, 0);
    for (int c : I)
      if (hr[(size_t)c] <= prm->tau_c * normA) { L.push_back(c); inL[(size_t)c] = 1; }
    for (int c = 0; c < pa; ++c)
      if (!inL[(size_t)c]) keep.push_back(c);
    rec[3] = (double)L.size();
    done = L.size() == I.size();
    if (!L.empty()) {
      std::vector<int32_t> idx(L.begin(), L.end());
      idx.insert(idx.end(), keep.begin(), keep.end());
      APF_CUDA(cudaMemcpyAsync(idxd.p, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
      const int32_t* dL = idxd.as<int32_t>();
      const int32_t* dK = dL + L.size();
      gather_columns<T>(ctx, n, (int64_t)L.size(), dL, Vh.as<T>(), ld, Vlock.as<T>() + nlock, ld);
      for (int c : L) lam_lock.push_back(hw[(size_t)c]);
      nlock += (int64_t)L.size();
      const int64_t nk = (int64_t)keep.size();
      if (nk > 0) {
        double* w2 = w + ld;
        gather_columns<T>(ctx, n, nk, dK, Vh.as<T>(), ld, X.as<T>(), ld);
        copy_block<T>(ctx, n, nk, X.as<T>(), ld, Vh.as<T>(), ld);
        gather_columns<T>(ctx, n, nk, dK, AVh.as<T>(), ld, X.as<T>(), ld);
        copy_block<T>(ctx, n, nk, X.as<T>(), ld, AVh.as<T>(), ld);
        gather_doubles(ctx, nk, dK, w, w2);
        APF_CUDA(cudaMemcpyAsync(w, w2, (size_t)nk * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
      }
      pa = nk;
      // the filter buffers' padding columns must stay zero: clear the tail
      if (pa < ld) {
        APF_CUDA(cudaMemset2DAsync(Vh.as<T>() + pa, ld * sizeof(T), 0, (size_t)(ld - pa) * sizeof(T), n, ctx->stream));
        APF_CUDA(cudaMemset2DAsync(AVh.as<T>() + pa, ld * sizeof(T), 0, (size_t)(ld - pa) * sizeof(T), n, ctx->stream));
      }
    }
    ki = k_next;
  }
};

// Locked pairs of the intervals (in the given order, each ascending) into the
// result, with their residuals recomputed from scratch.
template <class T>
static void assemble_result(apf_ctx* ctx, const apf_matrix* A, const std::vector<IntervalState<T>*>& ivs,
                            double normA, apf_result* out) {
  const int64_t n = A->n;
  int64_t e = 0;
  for (auto* s : ivs) e += (int64_t)s->lam_lock.size();
  out->ctx = ctx;
  out->n = n;
  out->e = e;
  out->dtype = A->dtype;
  out->lde = block_ld(e);
  out->lam.clear();
  out->res.assign((size_t)e, 0.0);
  out->vecs.alloc((size_t)n * out->lde * sizeof(T), ctx->stream, true);
  int64_t off = 0;
  for (auto* s : ivs) {
    const int64_t es = (int64_t)s->lam_lock.size();
    std::vector<int32_t> order((size_t)es);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t u, int32_t v) { return s->lam_lock[(size_t)u] < s->lam_lock[(size_t)v]; });
    for (int64_t j = 0; j < es; ++j) out->lam.push_back(s->lam_lock[(size_t)order[(size_t)j]]);
    if (es > 0) {
      DBuf od((size_t)es * sizeof(int32_t), ctx->stream, false);  // freed in stream order
      APF_CUDA(cudaMemcpyAsync(od.p, order.data(), (size_t)es * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
      gather_columns<T>(ctx, n, es, od.as<int32_t>(), s->Vlock.template as<T>(), s->ld, out->vecs.as<T>() + off, out->lde);
    }
    off += es;
  }
  if (e > 0) {
    DBuf lamd((size_t)e * sizeof(double), ctx->stream, false);
    APF_CUDA(cudaMemcpyAsync(lamd.p, out->lam.data(), (size_t)e * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    DBuf AVr((size_t)n * out->lde * sizeof(T), ctx->stream, true);
    spmm_plain<T>(ctx, A, out->vecs.as<T>(), out->lde, e, AVr.as<T>());
    DBuf rd((size_t)e * sizeof(double), ctx->stream, false);
    residual_norms<T>(ctx, n, e, AVr.as<T>(), out->vecs.as<T>(), out->lde, lamd.as<double>(), rd.as<double>(), nullptr, 0.0);
    APF_CUDA(cudaMemcpyAsync(out->res.data(), rd.p, (size_t)e * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    APF_CUDA(cudaStreamSynchronize(ctx->stream));
    for (auto& r : out->res) r /= normA;
  }
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
}

// ---- Sec. 3.4: eigenvalue counts and the subspace size ------------------------------------
// e~_s = (1/m) sum_c z_c^H rho_s(l(A)) z_c for every interval s, with rho_s its
// filter at the maximum degree and the same m real +-1 probes z_c for all.
// One batched filter application: the probe block is repeated once per
// interval, highest degree first.
template <class T>
static std::vector<double> count_estimates(apf_ctx* ctx, const apf_matrix* A, int precision, double l1, double l2,
                                           const std::vector<const std::vector<double>*>& coefs, int64_t m,
                                           uint64_t seed) {
  const int64_t n = A->n;
  const int64_t g = (int64_t)coefs.size();
  APF_REQUIRE(g >= 1 && m >= 1 && g * m <= 8 * APF_MAX_P, APF_ERR_ARG);
  std::vector<int> ord((size_t)g);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int u, int v) { return coefs[(size_t)u]->size() > coefs[(size_t)v]->size(); });
  std::vector<double> all;
  std::vector<int32_t> kc;
  std::vector<int64_t> coff;
  for (int s : ord) {
    const int64_t o = (int64_t)all.size();
    all.insert(all.end(), coefs[(size_t)s]->begin(), coefs[(size_t)s]->end());
    for (int64_t c = 0; c < m; ++c) {
      kc.push_back((int32_t)coefs[(size_t)s]->size() - 1);
      coff.push_back(o);
    }
  }
  const int64_t w = g * m, ld = block_ld(w);
  DBuf cd(all.size() * sizeof(double), ctx->stream, false);
  APF_CUDA(cudaMemcpyAsync(cd.p, all.data(), all.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  DBuf Z((size_t)n * ld * sizeof(T), ctx->stream, true), Y((size_t)n * ld * sizeof(T), ctx->stream, true);
  rademacher_block<T>(ctx, seed, 3u, n, m, g, Z.as<T>(), ld);
  FilterState<T> fs;
  fs.init(ctx, A, ld, l1, l2, std::vector<double>(), precision);
  FilterCount fc;
  fs.apply_cols(kc, coff, cd.as<double>(), Z.as<T>(), nullptr, nullptr, w, Y.as<T>(), nullptr, nullptr, &fc);
  DBuf dots((size_t)w * sizeof(double), ctx->stream, false);
  column_dots<T>(ctx, n, w, Z.as<T>(), Y.as<T>(), ld, dots.as<double>());
  std::vector<double> h((size_t)w);
  APF_CUDA(cudaMemcpyAsync(h.data(), dots.p, (size_t)w * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  if (fetch_device_error(ctx) != 0) throw ApfError{APF_ERR_TIMEOUT, "count estimate filter"};
  std::vector<double> e((size_t)g, 0.0);
  for (int64_t i = 0; i < g; ++i) {
    double s = 0.0;
    for (int64_t c = 0; c < m; ++c) s += h[(size_t)(i * m + c)];
    e[(size_t)ord[(size_t)i]] = s / (double)m;
  }
  return e;
}

// p = ceil(mu e~), e~ floored at 1, clipped to [1, min(n, APF_MAX_P)]
static int64_t subspace_size(double e_est, double mu, int64_t n) {
  const double want = ceil(mu * std::max(e_est, 1.0));
  int64_t p = want > (double)APF_MAX_P ? (int64_t)APF_MAX_P : (int64_t)want;
  p = std::min(p, n);
  return std::max<int64_t>(p, 1);
}

// ---- Alg. 4 ---------------------------------------------------------------------------
static double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) { cudaGetLastError(); return 0.0; }
  return (double)ms;
}

struct EventPool {
  std::vector<cudaEvent_t> ev;
  cudaEvent_t get() {
    cudaEvent_t e;
    APF_CUDA(cudaEventCreate(&e));
    ev.push_back(e);
    return e;
  }
  ~EventPool() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

struct IterEv { cudaEvent_t e0, e1, e2, e3, f0, f1; };

static void check_device_after_rr(apf_ctx* ctx) {
  const int derr = fetch_device_error(ctx);  // synchronises
  if (derr == DEV_EIGH_NOCONV) throw ApfError{APF_ERR_EIGH, "Rayleigh-Ritz eigensolver"};
  if (derr == DEV_BARRIER_TIMEOUT) throw ApfError{APF_ERR_TIMEOUT, "eigensolver barrier"};
  if (derr != 0) throw ApfError{APF_ERR_CUDA, "device error"};
}

static void finish_stats(apf_ctx* ctx, const std::vector<IterEv>& iev, const FilterCount& fc, int iters,
                         double deg_sum, apf_stats* st) {
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  for (auto& ev : iev) {
    st->ms_filter += elapsed_ms(ev.e0, ev.e1);
    st->ms_rr += elapsed_ms(ev.e1, ev.e2);
    st->ms_check += elapsed_ms(ev.e2, ev.e3);
    st->filter_kernel_ms += elapsed_ms(ev.f0, ev.f1);
  }
  st->iterations = iters;
  st->avg_degree = iters ? deg_sum / iters : 0.0;
  st->filter_launches = fc.launches;
  st->filter_steps = fc.steps;
  st->filter_bytes = fc.bytes;
  st->filter_step_bytes = fc.step_bytes;
  st->filter_kind = fc.kind;
  st->filter_g = fc.G;
  st->filter_vpt = fc.VPT;
  st->filter_graph_replays = fc.graph_replays;
}

struct Bounds {
  double lmin, lmax, l1, l2, normA;
};

static Bounds setup_bounds(apf_ctx* ctx, const apf_matrix* A, const apf_params* prm) {
  double bnd[6];
  spectrum_bounds(ctx, A, prm->lanczos_steps, prm->seed, prm->bound_pad, bnd);
  Bounds B;
  B.lmin = bnd[0];
  B.lmax = bnd[1];
  B.l1 = 2.0 / (B.lmax - B.lmin);
  B.l2 = -(B.lmax + B.lmin) / (B.lmax - B.lmin);
  // ||A|| of the convergence test (Sec. 4) from the unpadded Lanczos Ritz
  // values: they lie inside the spectrum, so this never exceeds the spectral
  // radius and ||r|| <= tau_c ||A|| holds for the true ||A|| at locking
  B.normA = std::max(fabs(bnd[2]), fabs(bnd[3]));
  return B;
}

}  // namespace apf
