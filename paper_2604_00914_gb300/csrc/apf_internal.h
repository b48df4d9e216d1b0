// Internal declarations of the apf library: context and matrix objects,
// device buffers, error handling and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "apf.h"
#include "scalar.cuh"

// ---- error handling: internal code throws, the C ABI catches ---------------
struct ApfError {
  apf_status status;
  std::string what;
};

#define APF_CUDA(call)                                                          \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      if (e_ == cudaErrorMemoryAllocation) throw ApfError{APF_ERR_OOM, #call}; \
      throw ApfError{APF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    }                                                                           \
  } while (0)

#define APF_REQUIRE(cond, status)                 \
  do {                                            \
    if (!(cond)) throw ApfError{status, #cond};   \
  } while (0)

// device-side error codes written to ctx->d_err (first writer wins)
enum DeviceError : int {
  DEV_OK = 0,
  DEV_CHOL_PIVOT = 1,
  DEV_EIGH_NOCONV = 2,
  DEV_BARRIER_TIMEOUT = 3,
  DEV_NONFINITE = 4
};

struct apf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  int* d_err = nullptr;          // device error word
  unsigned* d_bar = nullptr;     // grid-barrier words (count, generation)
  unsigned* d_counters = nullptr; // per-sweep rotation counters of the Jacobi solver
  int64_t launches = 0;          // kernels launched through this context
  double* h_pinned = nullptr;    // pinned staging buffer
  size_t h_pinned_bytes = 0;
  uint64_t wait_limit_ns = 0;    // device-side wait limit (apf_set_wait_limit); 0: the defaults below
  void* ws = nullptr;            // workspace of the tensor-core products (grown on demand)
  size_t ws_bytes = 0;
  std::string last_error;
};

// Time limits of the device-side waits: the filter kernels' mbarrier and
// two-step dependency waits (1 s), the eigensolver's grid barrier (2 s).
constexpr uint64_t kFilterWaitNs = 1000000000ull;
constexpr uint64_t kBarrierWaitNs = 2000000000ull;
inline uint64_t filter_wait_ns(const apf_ctx* c) { return c->wait_limit_ns ? c->wait_limit_ns : kFilterWaitNs; }
inline uint64_t barrier_wait_ns(const apf_ctx* c) { return c->wait_limit_ns ? c->wait_limit_ns : kBarrierWaitNs; }

struct apf_matrix {
  apf_ctx* ctx = nullptr;
  int64_t n = 0, nnz = 0;
  int dtype = APF_R64;
  int64_t* rowptr = nullptr;     // device, n + 1
  int32_t* colidx = nullptr;     // device, nnz (every row holds its diagonal)
  void* vals = nullptr;          // device, nnz values (double or double2)
  double gersh_lo = 0, gersh_hi = 0;  // Gershgorin interval
  // SELL-8 copy of the structure (rows in order, chunks of 8 rows padded to
  // their longest row); sell_src maps a slot to its CSR entry (-1: padding)
  bool sell_ok = false;
  int sell_lmax = 0;
  int64_t sell_slots = 0;
  int64_t* sell_chunk_ptr = nullptr;
  int32_t* sell_col = nullptr;
  int32_t* sell_src = nullptr;
  int64_t sell_bw = 0;           // max |i - j| (natural row order)
  int sell_halo = 0;             // near-row reach H of the column-tiled step with staged W rows (0: none)
  // a second SELL-8 copy in reverse Cuthill-McKee row order, for the two-step
  // filter pass (null when the natural order is already banded)
  int32_t* perm = nullptr;       // new -> old
  int32_t* iperm = nullptr;      // old -> new
  int64_t* psell_chunk_ptr = nullptr;
  int32_t* psell_col = nullptr;
  int32_t* psell_src = nullptr;
  int psell_lmax = 0;
  int64_t psell_slots = 0;
  int64_t psell_bw = 0;
  // autotuned Clenshaw-step shape per (element size, vectors per row):
  // value = kind * 10000 + G * 100 + VPT, kind 1 = SELL, 2 = SELL two-step, 4 / 5 = SELL column
  // tiles (5: near rows of W in shared memory), 0 = CSR
  std::vector<std::pair<int64_t, int>> tune_cache;
  // a pinned kernel (apf_matrix_set_filter_kernel): kind 0 = autotune
  int pin_kind = 0, pin_G = 0, pin_VPT = 0;
};

namespace apf {

// ---- device buffers (stream-ordered allocation) ----------------------------
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(size_t b, cudaStream_t st, bool zero = true) { alloc(b, st, zero); }
  void alloc(size_t b, cudaStream_t st, bool zero = true);
  void release();
  ~DBuf() { release(); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { p = o.p; bytes = o.bytes; s = o.s; o.p = nullptr; o.bytes = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; s = o.s; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
// leading dimension used for internal n x p blocks: a multiple of 8 elements
inline int64_t block_ld(int64_t p) { return round_up(p < 1 ? 1 : p, 8); }

void count_launch(apf_ctx* ctx, int k = 1);
void check_launch(apf_ctx* ctx);
// reads and clears the device error word (synchronises the stream)
int fetch_device_error(apf_ctx* ctx);

// ---- SpMM / Clenshaw step (k_spmm.cu) ---------------------------------------
// Out[i,:] = alpha (A W)[i,:] - Vin[i,:] + f .* Y[i,:]
//   f = coef_col[c] per column if coef_col != nullptr, else coef_scalar.
// Vin and Y may be null (terms dropped).  Out may alias Vin, never W.
// All blocks share leading dimension ld (elements, a multiple of the 16-byte
// vector width); ncols columns are computed (ncols <= ld, padded to the vector width).
template <class T, class TA>
void clenshaw_step(apf_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* colidx,
                   const TA* vals, const T* W, const T* Vin, const T* Y, int64_t ld,
                   int64_t ncols, const typename ScalarTraits<T>::Real* coef_col,
                   typename ScalarTraits<T>::Real coef_scalar,
                   typename ScalarTraits<T>::Real alpha, T* Out);

// SELL-8 form of the same step (A as sell_chunk_ptr / sell_col / sell values),
// with the given (G, VPT) shape; see spmm_sell.cuh.
template <class T, class TA>
void clenshaw_step_sell(apf_ctx* ctx, int G, int VPT, int64_t n, const int64_t* chunk_ptr,
                        const int32_t* scol, const TA* sval, int lmax, const T* W, const T* Vin,
                        const T* Y, int64_t ld, int64_t ncols,
                        const typename ScalarTraits<T>::Real* coef_col,
                        typename ScalarTraits<T>::Real coef_scalar,
                        typename ScalarTraits<T>::Real alpha, T* Out);
// The same step with the block cut into column tiles of G x VPT vectors, one
// tile per CTA (grid: row ranges x tiles); any width.  halo > 0: the rows of W
// within halo rows of a CTA's own come from shared memory.  See spmm_sell_ct.cuh.
template <class T, class TA>
void clenshaw_step_sell_ct(apf_ctx* ctx, int G, int VPT, int64_t n, const int64_t* chunk_ptr,
                           const int32_t* scol, const TA* sval, int lmax, const T* W, const T* Vin,
                           const T* Y, int64_t ld, int64_t ncols,
                           const typename ScalarTraits<T>::Real* coef_col,
                           typename ScalarTraits<T>::Real coef_scalar,
                           typename ScalarTraits<T>::Real alpha, T* Out, int halo);
// Two consecutive Clenshaw steps in one pass (SELL-8, temporal blocking):
// bufB = 2 A W - va + f1 Y with W = bufA, then bufA = 2 A bufB - bufA + f2 Y.
// bandwidth: max |i - j| of the stored pattern; seg_count / pass: see spmm_sell.cuh.
template <class T, class TA>
void clenshaw_sell_pair(apf_ctx* ctx, int G, int VPT, int64_t n, const int64_t* chunk_ptr,
                        const int32_t* scol, const TA* sval, int lmax, int64_t bandwidth, T* bufA,
                        T* bufB, const T* va, const T* Y, int64_t ld, int64_t ncols,
                        const typename ScalarTraits<T>::Real* coef1_col,
                        typename ScalarTraits<T>::Real coef1,
                        const typename ScalarTraits<T>::Real* coef2_col,
                        typename ScalarTraits<T>::Real coef2, unsigned* seg_count, unsigned pass);
// CSR form with an explicit (G, VPT) shape (0, 0: automatic choice)
template <class T, class TA>
void clenshaw_step_shape(apf_ctx* ctx, int G, int VPT, int64_t n, const int64_t* rowptr,
                         const int32_t* colidx, const TA* vals, const T* W, const T* Vin, const T* Y,
                         int64_t ld, int64_t ncols, const typename ScalarTraits<T>::Real* coef_col,
                         typename ScalarTraits<T>::Real coef_scalar,
                         typename ScalarTraits<T>::Real alpha, T* Out);
// vals_sell[s] = src[s] >= 0 ? vals_csr[src[s]] : 0
template <class TA>
void sell_gather_values(apf_ctx* ctx, int64_t slots, const int32_t* src, const TA* csr, TA* out);

// y = A x for one vector (Lanczos), FP64.
template <class T>
void spmv(apf_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* colidx, const T* vals,
          const T* x, T* y);

// vals_hat = s (l1 vals + l2 I) in FP64 or rounded to FP32 (TO = T or LowOf<T>)
template <class T, class TO>
void scale_shift_matrix(apf_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* colidx,
                        const T* vals, double l1, double l2, TO* out);

// Gershgorin interval of A (device reduction, result to host)
template <class T>
void gershgorin(apf_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* colidx,
                const T* vals, double* lo, double* hi);

// ---- dense tall-skinny products (k_dense.cu) ---------------------------------
// G (pa x pb, ldg) = X^H Y; X: n x pa (ldx), Y: n x pb (ldy).  hermitian: X == Y,
// only the upper tiles are computed and mirrored.
// the same product on the tensor cores, FP64-accurate by bf16 slicing (k_gram_tc.cu)
template <class T>
void gram_tc(apf_ctx* ctx, int64_t n, int64_t pa, int64_t pb, const T* X, int64_t ldx, const T* Y, int64_t ldy,
             T* G, int64_t ldg, bool hermitian);
template <class T>
void gram(apf_ctx* ctx, int64_t n, int64_t pa, int64_t pb, const T* X, int64_t ldx,
          const T* Y, int64_t ldy, T* G, int64_t ldg, bool hermitian);
// Z = beta Z0 + alpha X M on the tensor cores, FP64-accurate (k_oz_tc.cu)
template <class T>
void gemm_tall_tc(apf_ctx* ctx, int64_t n, int64_t pa, int64_t pb, const T* X, int64_t ldx, const T* M,
                  int64_t ldm, T* Z, int64_t ldz, double alpha, double beta, const T* Z0, int64_t ldz0);

// gram() with the split partials in caller-provided device scratch (no allocation)
template <class T>
void gram_scratch(cudaStream_t stream, int num_sms, int64_t n, int64_t pa, int64_t pb, const T* X,
                  int64_t ldx, const T* Y, int64_t ldy, T* G, int64_t ldg, void* scratch,
                  size_t scratch_bytes);

// Z (n x pb) = beta Z0 + alpha X M; X: n x pa, M: pa x pb (ldm).  Z may alias Z0.
// upper: M is upper triangular (rows below the diagonal are skipped).
template <class T>
void gemm_tall(apf_ctx* ctx, int64_t n, int64_t pa, int64_t pb, const T* X, int64_t ldx,
               const T* M, int64_t ldm, T* Z, int64_t ldz, double alpha, double beta,
               const T* Z0, int64_t ldz0, bool upper);

// C (m x n) = alpha op(A) op(B) + beta C for small matrices; op = 'N' or 'H'.
template <class T>
void small_gemm(apf_ctx* ctx, int64_t m, int64_t n, int64_t k, char opa, const T* A, int64_t lda,
                char opb, const T* B, int64_t ldb, T* C, int64_t ldc, double alpha, double beta);

// ---- small dense factorisations (k_small.cu) ---------------------------------
// In place: the upper triangle of G becomes R with G = R^H R (lower part zeroed).
// shift is added to the diagonal first.  Breakdown sets DEV_CHOL_PIVOT.
template <class T>
void cholesky_upper(apf_ctx* ctx, int64_t p, T* G, int64_t ldg, double shift);
// Rinv = R^{-1} for upper triangular R (p x p)
template <class T>
void tri_inv_upper(apf_ctx* ctx, int64_t p, const T* R, int64_t ldr, T* Rinv, int64_t ldri);
// Hermitian eigendecomposition by one-sided Jacobi; w ascending, U row-major.
template <class T>
void eigh_jacobi(apf_ctx* ctx, int64_t p, const T* B, int64_t ldb, double* w, T* U, int64_t ldu);
// B <- (B + B^H) / 2
template <class T>
void symmetrize(apf_ctx* ctx, int64_t p, T* B, int64_t ldb);
// infinity norm of a small matrix (device scalar out)
template <class T>
void small_inf_norm(apf_ctx* ctx, int64_t p, const T* B, int64_t ldb, double* out);

// ---- element-wise and reduction kernels (k_misc.cu) ----------------------------
template <class T>
void random_block(apf_ctx* ctx, uint64_t seed, uint32_t stream, int64_t n, int64_t p, T* X, int64_t ld);
// reps copies of an n x m block of +-1 side by side: X[i, r m + c] = -1 when
// the uniform draw of counter i m + c of (seed, stream) is below 1/2, else +1
template <class T>
void rademacher_block(apf_ctx* ctx, uint64_t seed, uint32_t stream, int64_t n, int64_t m, int64_t reps, T* X,
                      int64_t ld);
// out[c] = sum_i Re(conj(X[i, c]) Y[i, c]) in FP64 (device), c < p
template <class T>
void column_dots(apf_ctx* ctx, int64_t n, int64_t p, const T* X, const T* Y, int64_t ld, double* out);
template <class TI, class TO>
void cast_block(apf_ctx* ctx, int64_t n, int64_t p, const TI* X, int64_t ldx, TO* Y, int64_t ldy);
template <class T>
void copy_block(apf_ctx* ctx, int64_t n, int64_t p, const T* X, int64_t ldx, T* Y, int64_t ldy);
template <class T>
void scale_block(apf_ctx* ctx, int64_t n, int64_t p, double s, const T* X, int64_t ldx, T* Y, int64_t ldy);
// Y[:, c] = f[c] X[:, c] with coefficients f of X's real type (device); Y may equal X
template <class T>
void scale_columns(apf_ctx* ctx, int64_t n, int64_t p, const typename ScalarTraits<T>::Real* f, const T* X,
                   int64_t ld, T* Y);
// per-column coefficients of a batched (multi-slice) filter; see k_misc.cu
template <class TF>
void coef_columns(apf_ctx* ctx, int64_t p, int64_t ld, int K, const double* coef, const int64_t* coff,
                  const int32_t* kc, const double* lam, double l1, double l2, TF* F, double* rho);
// per-column partial sums of |AV - w V|^2 -> res[p] = sqrt (device); optionally
// Rout = l1 (AV - w V) rounded to FP32 (for the defect filter)
template <class T>
void residual_norms(apf_ctx* ctx, int64_t n, int64_t p, const T* AV, const T* V, int64_t ld,
                    const double* w, double* res, typename LowOf<T>::type* Rout, double l1,
                    const int32_t* rout_rows = nullptr);  // Rout row i goes to row rout_rows[i]
// per-column Clenshaw coefficients of the defect recurrence and rho(mu_c)
void defect_coefficients(apf_ctx* ctx, int64_t p, int64_t ld, int k, const double* coef_dev,
                         const double* lam, double l1, double l2, float* F, double* rho);
// X = V diag(rho) + hi(D)
template <class T>
void defect_combine(apf_ctx* ctx, int64_t n, int64_t p, const T* V, int64_t ldv, const double* rho,
                    const typename LowOf<T>::type* D, int64_t ldd, T* X, int64_t ldx,
                    const int32_t* d_rows = nullptr);  // row i of X takes row d_rows[i] of D
// Y[i, :] = X[src_rows[i], :] converted (src_rows null: plain cast)
template <class TI, class TO>
void cast_block_rows(apf_ctx* ctx, int64_t n, int64_t p, const TI* X, int64_t ldx, TO* Y, int64_t ldy,
                     const int32_t* src_rows);
// Y[:, j] = X[:, idx[j]], j < m  (idx on device)
template <class T>
void gather_columns(apf_ctx* ctx, int64_t n, int64_t m, const int32_t* idx, const T* X, int64_t ldx,
                    T* Y, int64_t ldy);
// dst (col-major, ldd) = src (row-major n x p, lds)
template <class T>
void to_col_major(apf_ctx* ctx, int64_t n, int64_t p, const T* src, int64_t lds, T* dst, int64_t ldd);
// gather vector entries w_out[j] = w[idx[j]]
void gather_doubles(apf_ctx* ctx, int64_t m, const int32_t* idx, const double* w, double* out);

// Lanczos helpers on contiguous vectors
template <class T>
void dot_many(apf_ctx* ctx, int64_t n, int64_t m, const T* Q, const T* w, T* out);  // out[j] = Q_j^H w
template <class T>
void axpy_many(apf_ctx* ctx, int64_t n, int64_t m, const T* Q, const T* c, T* w);   // w -= sum_j c_j Q_j
template <class T>
void norm2(apf_ctx* ctx, int64_t n, const T* x, double* out);                        // out = ||x||
template <class T>
void scale_vec_by_inv(apf_ctx* ctx, int64_t n, const T* x, const double* s, T* y);  // y = x / s
template <class T>
void lanczos_update(apf_ctx* ctx, int64_t n, int j, const T* Q, T* w, double* alpha,
                    const double* beta);  // alpha_j = Re q_j^H w; w -= alpha_j q_j + beta_{j-1} q_{j-1}

// ---- solver (solver.cu) --------------------------------------------------------
void spectrum_bounds(apf_ctx* ctx, const apf_matrix* A, int steps, uint64_t seed, double pad,
                     double out[6]);

}  // namespace apf
