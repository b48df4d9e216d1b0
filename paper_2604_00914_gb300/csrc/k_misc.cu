// Element-wise and reduction kernels around the filter and the Ritz step:
// seeded random blocks (SplitMix64), precision casts, residual norms (the
// residual step of Alg. 4), the per-column coefficients and recombination of
// the defect form of the filter, column compaction for locking (Alg. 4),
// and the vector kernels of the Lanczos bound estimate (Sec. 3.4).
#include "apf_internal.h"

namespace apf {

// ---- context helpers and device buffers ------------------------------------------
void DBuf::alloc(size_t b, cudaStream_t st, bool zero) {
  release();
  s = st;
  bytes = b;
  if (b == 0) return;
  APF_CUDA(cudaMallocAsync(&p, b, st));
  if (zero) APF_CUDA(cudaMemsetAsync(p, 0, b, st));
}

void DBuf::release() {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
  bytes = 0;
}

void count_launch(apf_ctx* ctx, int k) {
  ctx->launches += k;
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw ApfError{APF_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e)};
  }
}

void check_launch(apf_ctx* ctx) { count_launch(ctx, 0); }

int fetch_device_error(apf_ctx* ctx) {
  int h = 0;
  APF_CUDA(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  if (h != 0) APF_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  return h;
}

static inline unsigned grid1d(int64_t n, int t = 256) {
  int64_t g = (n + t - 1) / t;
  return (unsigned)(g < 1 ? 1 : g);
}

// ---- SplitMix64, counter form (Steele, Lea and Flood, OOPSLA 2014) ------------------
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double sm64_uniform(uint64_t key, uint64_t i) {
  const uint64_t z = sm64_mix(key + 0x9E3779B97F4A7C15ull * (i + 1));
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

template <class T>
__global__ void k_random_block(uint64_t key, int64_t n, int64_t p, T* X, int64_t ld) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * p) return;
  const int64_t i = e / p, c = e % p;
  if constexpr (ScalarTraits<T>::is_complex) {
    const double re = 2.0 * sm64_uniform(key, 2 * (uint64_t)e) - 1.0;
    const double im = 2.0 * sm64_uniform(key, 2 * (uint64_t)e + 1) - 1.0;
    X[i * ld + c] = make_val<T>(re, im);
  } else {
    X[i * ld + c] = make_val<T>(2.0 * sm64_uniform(key, (uint64_t)e) - 1.0, 0.0);
  }
}

static uint64_t host_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <class T>
void random_block(apf_ctx* ctx, uint64_t seed, uint32_t stream, int64_t n, int64_t p, T* X, int64_t ld) {
  if (n * p == 0) return;
  const uint64_t key = host_mix(seed + 0x9E3779B97F4A7C15ull * ((uint64_t)stream + 1));
  k_random_block<T><<<grid1d(n * p), 256, 0, ctx->stream>>>(key, n, p, X, ld);
  count_launch(ctx);
}
template void random_block<double>(apf_ctx*, uint64_t, uint32_t, int64_t, int64_t, double*, int64_t);
template void random_block<double2>(apf_ctx*, uint64_t, uint32_t, int64_t, int64_t, double2*, int64_t);

template <class T>
__global__ void k_rademacher_block(uint64_t key, int64_t n, int64_t m, int64_t reps, T* X, int64_t ld) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m * reps) return;
  const int64_t i = e / (m * reps), col = e % (m * reps), c = col % m;
  const double u = sm64_uniform(key, (uint64_t)(i * m + c));
  X[i * ld + col] = make_val<T>(u < 0.5 ? -1.0 : 1.0, 0.0);
}

template <class T>
void rademacher_block(apf_ctx* ctx, uint64_t seed, uint32_t stream, int64_t n, int64_t m, int64_t reps, T* X,
                      int64_t ld) {
  if (n * m * reps == 0) return;
  const uint64_t key = host_mix(seed + 0x9E3779B97F4A7C15ull * ((uint64_t)stream + 1));
  k_rademacher_block<T><<<grid1d(n * m * reps), 256, 0, ctx->stream>>>(key, n, m, reps, X, ld);
  count_launch(ctx);
}
template void rademacher_block<double>(apf_ctx*, uint64_t, uint32_t, int64_t, int64_t, int64_t, double*, int64_t);
template void rademacher_block<double2>(apf_ctx*, uint64_t, uint32_t, int64_t, int64_t, int64_t, double2*, int64_t);

// ---- casts and copies -----------------------------------------------------------------
__device__ __forceinline__ float cvt(double v, float*) { return (float)v; }
__device__ __forceinline__ float2 cvt(double2 v, float2*) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double cvt(float v, double*) { return (double)v; }
__device__ __forceinline__ double2 cvt(float2 v, double2*) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double cvt(double v, double*) { return v; }
__device__ __forceinline__ double2 cvt(double2 v, double2*) { return v; }

template <class TI, class TO>
__global__ void k_cast(int64_t n, int64_t p, const TI* __restrict__ X, int64_t ldx, TO* __restrict__ Y,
                       int64_t ldy) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * p) return;
  const int64_t i = e / p, c = e % p;
  Y[i * ldy + c] = cvt(X[i * ldx + c], (TO*)nullptr);
}

template <class TI, class TO>
void cast_block(apf_ctx* ctx, int64_t n, int64_t p, const TI* X, int64_t ldx, TO* Y, int64_t ldy) {
  if (n * p == 0) return;
  k_cast<TI, TO><<<grid1d(n * p), 256, 0, ctx->stream>>>(n, p, X, ldx, Y, ldy);
  count_launch(ctx);
}
template void cast_block<double, float>(apf_ctx*, int64_t, int64_t, const double*, int64_t, float*, int64_t);
template void cast_block<double2, float2>(apf_ctx*, int64_t, int64_t, const double2*, int64_t, float2*, int64_t);
template void cast_block<float, double>(apf_ctx*, int64_t, int64_t, const float*, int64_t, double*, int64_t);
template void cast_block<float2, double2>(apf_ctx*, int64_t, int64_t, const float2*, int64_t, double2*, int64_t);

// Y[i, :] = X[src[i], :] converted (a row gather between orderings)
template <class TI, class TO>
__global__ void k_cast_rows(int64_t n, int64_t p, const TI* __restrict__ X, int64_t ldx, TO* __restrict__ Y,
                            int64_t ldy, const int32_t* __restrict__ src) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * p) return;
  const int64_t i = e / p, c = e % p;
  Y[i * ldy + c] = cvt(X[(int64_t)src[i] * ldx + c], (TO*)nullptr);
}

template <class TI, class TO>
void cast_block_rows(apf_ctx* ctx, int64_t n, int64_t p, const TI* X, int64_t ldx, TO* Y, int64_t ldy,
                     const int32_t* src_rows) {
  if (!src_rows) {
    cast_block<TI, TO>(ctx, n, p, X, ldx, Y, ldy);
    return;
  }
  if (n * p == 0) return;
  k_cast_rows<TI, TO><<<grid1d(n * p), 256, 0, ctx->stream>>>(n, p, X, ldx, Y, ldy, src_rows);
  count_launch(ctx);
}
template void cast_block_rows<double, float>(apf_ctx*, int64_t, int64_t, const double*, int64_t, float*, int64_t, const int32_t*);
template void cast_block_rows<double2, float2>(apf_ctx*, int64_t, int64_t, const double2*, int64_t, float2*, int64_t, const int32_t*);
template void cast_block_rows<float, double>(apf_ctx*, int64_t, int64_t, const float*, int64_t, double*, int64_t, const int32_t*);
template void cast_block_rows<float2, double2>(apf_ctx*, int64_t, int64_t, const float2*, int64_t, double2*, int64_t, const int32_t*);

template <class T>
void copy_block(apf_ctx* ctx, int64_t n, int64_t p, const T* X, int64_t ldx, T* Y, int64_t ldy) {
  if (n * p == 0) return;
  if (ldx == p && ldy == p) {
    APF_CUDA(cudaMemcpyAsync(Y, X, (size_t)n * p * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream));
    return;
  }
  APF_CUDA(cudaMemcpy2DAsync(Y, ldy * sizeof(T), X, ldx * sizeof(T), p * sizeof(T), n,
                             cudaMemcpyDeviceToDevice, ctx->stream));
}
template void copy_block<double>(apf_ctx*, int64_t, int64_t, const double*, int64_t, double*, int64_t);
template void copy_block<double2>(apf_ctx*, int64_t, int64_t, const double2*, int64_t, double2*, int64_t);
template void copy_block<float>(apf_ctx*, int64_t, int64_t, const float*, int64_t, float*, int64_t);
template void copy_block<float2>(apf_ctx*, int64_t, int64_t, const float2*, int64_t, float2*, int64_t);

template <class T>
__global__ void k_scale_block(int64_t n, int64_t p, double s, const T* __restrict__ X, int64_t ldx,
                              T* __restrict__ Y, int64_t ldy) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * p) return;
  const int64_t i = e / p, c = e % p;
  Y[i * ldy + c] = rmul((typename ScalarTraits<T>::Real)s, X[i * ldx + c]);
}

template <class T>
void scale_block(apf_ctx* ctx, int64_t n, int64_t p, double s, const T* X, int64_t ldx, T* Y, int64_t ldy) {
  if (n * p == 0) return;
  k_scale_block<T><<<grid1d(n * p), 256, 0, ctx->stream>>>(n, p, s, X, ldx, Y, ldy);
  count_launch(ctx);
}
template void scale_block<double>(apf_ctx*, int64_t, int64_t, double, const double*, int64_t, double*, int64_t);
template void scale_block<double2>(apf_ctx*, int64_t, int64_t, double, const double2*, int64_t, double2*, int64_t);
template void scale_block<float>(apf_ctx*, int64_t, int64_t, double, const float*, int64_t, float*, int64_t);
template void scale_block<float2>(apf_ctx*, int64_t, int64_t, double, const float2*, int64_t, float2*, int64_t);

// per-column scaling Y[:, c] = f[c] X[:, c] (f on device, coefficients of X's real type)
template <class T>
__global__ void k_scale_cols(int64_t n, int64_t p, const typename ScalarTraits<T>::Real* __restrict__ f,
                             const T* __restrict__ X, int64_t ld, T* __restrict__ Y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * p) return;
  const int64_t i = e / p, c = e % p;
  Y[i * ld + c] = rmul(f[c], X[i * ld + c]);
}

template <class T>
void scale_columns(apf_ctx* ctx, int64_t n, int64_t p, const typename ScalarTraits<T>::Real* f, const T* X,
                   int64_t ld, T* Y) {
  if (n * p == 0) return;
  k_scale_cols<T><<<grid1d(n * p), 256, 0, ctx->stream>>>(n, p, f, X, ld, Y);
  count_launch(ctx);
}
template void scale_columns<float>(apf_ctx*, int64_t, int64_t, const float*, const float*, int64_t, float*);
template void scale_columns<float2>(apf_ctx*, int64_t, int64_t, const float*, const float2*, int64_t, float2*);
template void scale_columns<double>(apf_ctx*, int64_t, int64_t, const double*, const double*, int64_t, double*);
template void scale_columns<double2>(apf_ctx*, int64_t, int64_t, const double*, const double2*, int64_t, double2*);

// Per-column coefficients of a batched filter (spectrum slices): column c uses
// the coefficient vector coef + coff[c] of degree kc[c], zero above it, inside
// a recurrence of global degree K.  Plain form (lam == nullptr): F[j][c] = a_j.
// Defect form: the column's scalar Clenshaw sequence beta_j(mu_c),
// mu_c = l1 lam_c + l2, gives F[j][c] = 2 beta_{j+1} (0 < j < K), F[0][c] =
// beta_1 and rho_c = a_0 + mu beta_1 - beta_2.  Padding columns get zeros.
template <class TF>
__global__ void k_coef_columns(int64_t p, int64_t ld, int K, const double* __restrict__ coef,
                               const int64_t* __restrict__ coff, const int32_t* __restrict__ kc,
                               const double* __restrict__ lam, double l1, double l2, TF* __restrict__ F,
                               double* __restrict__ rho) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ld) return;
  if (c >= p) {
    for (int j = 0; j <= K; ++j) F[(int64_t)j * ld + c] = (TF)0;
    if (rho) rho[c] = 0.0;
    return;
  }
  const double* a = coef + coff[c];
  const int k = kc[c];
  if (!lam) {
    for (int j = 0; j <= K; ++j) F[(int64_t)j * ld + c] = (TF)(j <= k ? a[j] : 0.0);
    return;
  }
  const double mu = l1 * lam[c] + l2;
  double b1 = 0.0, b2 = 0.0;  // beta_{j+1}, beta_{j+2}
  F[(int64_t)K * ld + c] = (TF)0;
  for (int j = K; j >= 1; --j) {
    const double aj = j <= k ? a[j] : 0.0;
    const double bj = aj + 2.0 * mu * b1 - b2;
    if (j < K) F[(int64_t)j * ld + c] = (TF)(2.0 * b1);
    b2 = b1;
    b1 = bj;
  }
  F[c] = (TF)b1;
  rho[c] = a[0] + mu * b1 - b2;
}

template <class TF>
void coef_columns(apf_ctx* ctx, int64_t p, int64_t ld, int K, const double* coef, const int64_t* coff,
                  const int32_t* kc, const double* lam, double l1, double l2, TF* F, double* rho) {
  k_coef_columns<TF><<<grid1d(ld, 128), 128, 0, ctx->stream>>>(p, ld, K, coef, coff, kc, lam, l1, l2, F, rho);
  count_launch(ctx);
}
template void coef_columns<float>(apf_ctx*, int64_t, int64_t, int, const double*, const int64_t*, const int32_t*,
                                  const double*, double, double, float*, double*);
template void coef_columns<double>(apf_ctx*, int64_t, int64_t, int, const double*, const int64_t*, const int32_t*,
                                   const double*, double, double, double*, double*);

// ---- residual norms ||A v_c - w_c v_c|| (and the mapped residual in FP32) -------------
template <class T>
__global__ void k_residual_partial(int64_t n, int64_t p, const T* __restrict__ AV,
                                   const T* __restrict__ V, int64_t ld, const double* __restrict__ w,
                                   int64_t rows_per_block, double* __restrict__ part,
                                   typename LowOf<T>::type* Rout, double l1,
                                   const int32_t* __restrict__ rout_rows) {
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
  const int64_t r1 = min(n, r0 + rows_per_block);
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p) return;
  const double wc = w[c];
  double s = 0.0;
  for (int64_t i = r0; i < r1; ++i) {
    const T r = sub(AV[i * ld + c], rmul(wc, V[i * ld + c]));
    s += abs2(r);
    if (Rout) Rout[(rout_rows ? (int64_t)rout_rows[i] : i) * ld + c] = to_lo(rmul(l1, r));
  }
  part[(int64_t)blockIdx.y * p + c] = s;
}

// partial sums of Re(conj(x) y) per column over a band of rows
template <class T>
__global__ void k_dot_partial(int64_t n, int64_t p, const T* __restrict__ X, const T* __restrict__ Y, int64_t ld,
                              int64_t rows_per_block, double* __restrict__ part) {
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
  const int64_t r1 = min(n, r0 + rows_per_block);
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p) return;
  double s = 0.0;
  for (int64_t i = r0; i < r1; ++i) s += re_dot(X[i * ld + c], Y[i * ld + c]);
  part[(int64_t)blockIdx.y * p + c] = s;
}

__global__ void k_colsum(int64_t p, int64_t nb, const double* __restrict__ part, double* __restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p) return;
  double s = 0.0;
  for (int64_t b = 0; b < nb; ++b) s += part[b * p + c];
  out[c] = s;
}

__global__ void k_colsum_sqrt(int64_t p, int64_t nb, const double* __restrict__ part, double* __restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p) return;
  double s = 0.0;
  for (int64_t b = 0; b < nb; ++b) s += part[b * p + c];
  out[c] = sqrt(s);
}

template <class T>
void residual_norms(apf_ctx* ctx, int64_t n, int64_t p, const T* AV, const T* V, int64_t ld,
                    const double* w, double* res, typename LowOf<T>::type* Rout, double l1,
                    const int32_t* rout_rows) {
  if (p == 0) return;
  const int64_t cb = (p + 127) / 128;
  int64_t nb = (4LL * ctx->num_sms + cb - 1) / cb;
  if (nb > n) nb = n;
  if (nb < 1) nb = 1;
  const int64_t rows = (n + nb - 1) / nb;
  nb = (n + rows - 1) / rows;
  if (nb < 1) nb = 1;
  DBuf part((size_t)nb * p * sizeof(double), ctx->stream, true);
  dim3 grid((unsigned)cb, (unsigned)nb);
  k_residual_partial<T><<<grid, 128, 0, ctx->stream>>>(n, p, AV, V, ld, w, rows, part.as<double>(), Rout, l1,
                                                       rout_rows);
  k_colsum_sqrt<<<grid1d(p, 128), 128, 0, ctx->stream>>>(p, nb, part.as<double>(), res);
  count_launch(ctx, 2);
}
template void residual_norms<double>(apf_ctx*, int64_t, int64_t, const double*, const double*, int64_t,
                                     const double*, double*, float*, double, const int32_t*);
template void residual_norms<double2>(apf_ctx*, int64_t, int64_t, const double2*, const double2*, int64_t,
                                      const double*, double*, float2*, double, const int32_t*);

template <class T>
void column_dots(apf_ctx* ctx, int64_t n, int64_t p, const T* X, const T* Y, int64_t ld, double* out) {
  if (p == 0) return;
  const int64_t cb = (p + 127) / 128;
  int64_t nb = (4LL * ctx->num_sms + cb - 1) / cb;
  if (nb > n) nb = n;
  if (nb < 1) nb = 1;
  const int64_t rows = (n + nb - 1) / nb;
  nb = (n + rows - 1) / rows;
  if (nb < 1) nb = 1;
  DBuf part((size_t)nb * p * sizeof(double), ctx->stream, true);
  k_dot_partial<T><<<dim3((unsigned)cb, (unsigned)nb), 128, 0, ctx->stream>>>(n, p, X, Y, ld, rows, part.as<double>());
  k_colsum<<<grid1d(p, 128), 128, 0, ctx->stream>>>(p, nb, part.as<double>(), out);
  count_launch(ctx, 2);
}
template void column_dots<double>(apf_ctx*, int64_t, int64_t, const double*, const double*, int64_t, double*);
template void column_dots<double2>(apf_ctx*, int64_t, int64_t, const double2*, const double2*, int64_t, double*);

// ---- the defect form of the filter -------------------------------------------------------
// Column c with mu = l1 lam_c + l2 runs the scalar Clenshaw recurrence
// beta_j = a_j + 2 mu beta_{j+1} - beta_{j+2} (j = k..1).  The block recurrence
// for D is driven by R_hat = A_hat V - V diag(mu) with coefficient 2 beta_{j+1}
// at step j (stored in F[j]) and beta_1 at the last step (F[0]);
// rho_c = a_0 + mu beta_1 - beta_2 is rho(l(lam_c)).
__global__ void k_defect_coef(int64_t p, int64_t ld, int k, const double* __restrict__ a,
                              const double* __restrict__ lam, double l1, double l2,
                              float* __restrict__ F, double* __restrict__ rho) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ld) return;
  if (c >= p) {
    for (int j = 0; j <= k; ++j) F[(int64_t)j * ld + c] = 0.0f;
    return;
  }
  const double mu = l1 * lam[c] + l2;
  double b1 = 0.0, b2 = 0.0;  // beta_{j+1}, beta_{j+2}
  F[(int64_t)k * ld + c] = 0.0f;
  for (int j = k; j >= 1; --j) {
    const double bj = a[j] + 2.0 * mu * b1 - b2;
    if (j < k) F[(int64_t)j * ld + c] = (float)(2.0 * b1);
    b2 = b1;
    b1 = bj;
  }
  F[c] = (float)b1;
  rho[c] = a[0] + mu * b1 - b2;
}

void defect_coefficients(apf_ctx* ctx, int64_t p, int64_t ld, int k, const double* coef_dev,
                         const double* lam, double l1, double l2, float* F, double* rho) {
  k_defect_coef<<<grid1d(ld, 128), 128, 0, ctx->stream>>>(p, ld, k, coef_dev, lam, l1, l2, F, rho);
  count_launch(ctx);
}

template <class T>
__global__ void k_defect_combine(int64_t n, int64_t p, const T* __restrict__ V, int64_t ldv,
                                 const double* __restrict__ rho,
                                 const typename LowOf<T>::type* __restrict__ D, int64_t ldd,
                                 T* __restrict__ X, int64_t ldx, const int32_t* __restrict__ d_rows) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * p) return;
  const int64_t i = e / p, c = e % p;
  T v = rmul(rho[c], V[i * ldv + c]);
  if (D) v = add(v, to_hi(D[(d_rows ? (int64_t)d_rows[i] : i) * ldd + c]));
  X[i * ldx + c] = v;
}

template <class T>
void defect_combine(apf_ctx* ctx, int64_t n, int64_t p, const T* V, int64_t ldv, const double* rho,
                    const typename LowOf<T>::type* D, int64_t ldd, T* X, int64_t ldx, const int32_t* d_rows) {
  if (n * p == 0) return;
  k_defect_combine<T><<<grid1d(n * p), 256, 0, ctx->stream>>>(n, p, V, ldv, rho, D, ldd, X, ldx, d_rows);
  count_launch(ctx);
}
template void defect_combine<double>(apf_ctx*, int64_t, int64_t, const double*, int64_t, const double*,
                                     const float*, int64_t, double*, int64_t, const int32_t*);
template void defect_combine<double2>(apf_ctx*, int64_t, int64_t, const double2*, int64_t, const double*,
                                      const float2*, int64_t, double2*, int64_t, const int32_t*);

// ---- column gathers and layout changes ----------------------------------------------------
template <class T>
__global__ void k_gather_cols(int64_t n, int64_t m, const int32_t* __restrict__ idx,
                              const T* __restrict__ X, int64_t ldx, T* __restrict__ Y, int64_t ldy) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  const int64_t i = e / m, j = e % m;
  Y[i * ldy + j] = X[i * ldx + idx[j]];
}

template <class T>
void gather_columns(apf_ctx* ctx, int64_t n, int64_t m, const int32_t* idx, const T* X, int64_t ldx,
                    T* Y, int64_t ldy) {
  if (n * m == 0) return;
  k_gather_cols<T><<<grid1d(n * m), 256, 0, ctx->stream>>>(n, m, idx, X, ldx, Y, ldy);
  count_launch(ctx);
}
template void gather_columns<double>(apf_ctx*, int64_t, int64_t, const int32_t*, const double*, int64_t,
                                     double*, int64_t);
template void gather_columns<double2>(apf_ctx*, int64_t, int64_t, const int32_t*, const double2*, int64_t,
                                      double2*, int64_t);

template <class T>
__global__ void k_to_colmajor(int64_t n, int64_t p, const T* __restrict__ src, int64_t lds,
                              T* __restrict__ dst, int64_t ldd) {
  __shared__ T tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r, c = c0 + threadIdx.x;
    if (i < n && c < p) tile[r][threadIdx.x] = src[i * lds + c];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t c = c0 + r, i = i0 + threadIdx.x;
    if (i < n && c < p) dst[c * ldd + i] = tile[threadIdx.x][r];
  }
}

template <class T>
void to_col_major(apf_ctx* ctx, int64_t n, int64_t p, const T* src, int64_t lds, T* dst, int64_t ldd) {
  if (n * p == 0) return;
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((p + 31) / 32)), block(32, 8);
  k_to_colmajor<T><<<grid, block, 0, ctx->stream>>>(n, p, src, lds, dst, ldd);
  count_launch(ctx);
}
template void to_col_major<double>(apf_ctx*, int64_t, int64_t, const double*, int64_t, double*, int64_t);
template void to_col_major<double2>(apf_ctx*, int64_t, int64_t, const double2*, int64_t, double2*, int64_t);

__global__ void k_gather_d(int64_t m, const int32_t* __restrict__ idx, const double* __restrict__ w,
                           double* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) out[j] = w[idx[j]];
}

void gather_doubles(apf_ctx* ctx, int64_t m, const int32_t* idx, const double* w, double* out) {
  if (m == 0) return;
  k_gather_d<<<grid1d(m), 256, 0, ctx->stream>>>(m, idx, w, out);
  count_launch(ctx);
}

// ---- Lanczos vector kernels (vectors contiguous, basis Q column j at Q + j n) -------------
template <class T>
__global__ void k_dot_many(int64_t n, const T* __restrict__ Q, const T* __restrict__ w, T* __restrict__ out) {
  __shared__ T red[32];
  const T* q = Q + (int64_t)blockIdx.x * n;
  T s = szero<T>();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) madd_conj(s, q[i], w[i]);
  s = warp_sum(s);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    T v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : szero<T>();
    v = warp_sum(v);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

template <class T>
void dot_many(apf_ctx* ctx, int64_t n, int64_t m, const T* Q, const T* w, T* out) {
  if (m == 0) return;
  k_dot_many<T><<<(unsigned)m, 1024, 0, ctx->stream>>>(n, Q, w, out);
  count_launch(ctx);
}
template void dot_many<double>(apf_ctx*, int64_t, int64_t, const double*, const double*, double*);
template void dot_many<double2>(apf_ctx*, int64_t, int64_t, const double2*, const double2*, double2*);

template <class T>
__global__ void k_axpy_many(int64_t n, int64_t m, const T* __restrict__ Q, const T* __restrict__ c, T* w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T s = w[i];
  for (int64_t j = 0; j < m; ++j) s = sub(s, mul(Q[j * n + i], c[j]));
  w[i] = s;
}

template <class T>
void axpy_many(apf_ctx* ctx, int64_t n, int64_t m, const T* Q, const T* c, T* w) {
  if (m == 0 || n == 0) return;
  k_axpy_many<T><<<grid1d(n), 256, 0, ctx->stream>>>(n, m, Q, c, w);
  count_launch(ctx);
}
template void axpy_many<double>(apf_ctx*, int64_t, int64_t, const double*, const double*, double*);
template void axpy_many<double2>(apf_ctx*, int64_t, int64_t, const double2*, const double2*, double2*);

template <class T>
__global__ void k_norm_partial(int64_t n, const T* __restrict__ x, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += abs2(x[i]);
  s = warp_sum(s);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__global__ void k_sum_sqrt(int nb, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b];
  s = warp_sum(s);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) out[0] = sqrt(v);
  }
}

template <class T>
void norm2(apf_ctx* ctx, int64_t n, const T* x, double* out) {
  int nb = (int)((n + 1023) / 1024);
  if (nb > 2 * ctx->num_sms) nb = 2 * ctx->num_sms;
  if (nb < 1) nb = 1;
  DBuf part((size_t)nb * sizeof(double), ctx->stream, false);
  k_norm_partial<T><<<nb, 1024, 0, ctx->stream>>>(n, x, part.as<double>());
  k_sum_sqrt<<<1, 1024, 0, ctx->stream>>>(nb, part.as<double>(), out);
  count_launch(ctx, 2);
}
template void norm2<double>(apf_ctx*, int64_t, const double*, double*);
template void norm2<double2>(apf_ctx*, int64_t, const double2*, double*);

template <class T>
__global__ void k_scale_inv(int64_t n, const T* __restrict__ x, const double* __restrict__ s, T* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = rmul(1.0 / s[0], x[i]);
}

template <class T>
void scale_vec_by_inv(apf_ctx* ctx, int64_t n, const T* x, const double* s, T* y) {
  if (n == 0) return;
  k_scale_inv<T><<<grid1d(n), 256, 0, ctx->stream>>>(n, x, s, y);
  count_launch(ctx);
}
template void scale_vec_by_inv<double>(apf_ctx*, int64_t, const double*, const double*, double*);
template void scale_vec_by_inv<double2>(apf_ctx*, int64_t, const double2*, const double*, double2*);

// alpha_j = Re(q_j^H w) from the dot stored in dotv; w -= alpha_j q_j + beta_{j-1} q_{j-1}
template <class T>
__global__ void k_lanczos_axpy(int64_t n, int j, const T* __restrict__ Q, T* __restrict__ w,
                               const T* __restrict__ dotv, double* __restrict__ alpha,
                               const double* __restrict__ beta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double a = real_(dotv[0]);
  if (i == 0) alpha[j] = a;
  if (i >= n) return;
  T v = sub(w[i], rmul(a, Q[(int64_t)j * n + i]));
  if (j > 0) v = sub(v, rmul(beta[j - 1], Q[(int64_t)(j - 1) * n + i]));
  w[i] = v;
}

template <class T>
void lanczos_update(apf_ctx* ctx, int64_t n, int j, const T* Q, T* w, double* alpha, const double* beta) {
  // alpha lives in a scratch slot after the dot product
  DBuf d(sizeof(T), ctx->stream, false);
  dot_many<T>(ctx, n, 1, Q + (int64_t)j * n, w, d.as<T>());
  k_lanczos_axpy<T><<<grid1d(n), 256, 0, ctx->stream>>>(n, j, Q, w, d.as<T>(), alpha, beta);
  count_launch(ctx);
}
template void lanczos_update<double>(apf_ctx*, int64_t, int, const double*, double*, double*, const double*);
template void lanczos_update<double2>(apf_ctx*, int64_t, int, const double2*, double2*, double*, const double*);

}  // namespace apf
