// Dense FP64 / complex-FP64 products of the orthogonalisation and
// Rayleigh-Ritz steps of Alg. 4:
//   gram       G = X^H Y        (n x pa)^H (n x pb), n >> pa, pb
//   gemm_tall  Z = b Z0 + a X M (n x pa) (pa x pb)
//   small_gemm C = a op(A) op(B) + b C   for p x p matrices
// The tall products split the long dimension n across CTAs; the Gram writes
// per-CTA partial tiles that a second kernel sums in a fixed order, so the
// result does not depend on scheduling.
#include "apf_internal.h"

namespace apf {

constexpr int GT = 32;   // Gram output tile (GT x GT), 2 x 2 per thread
constexpr int GRK = 32;  // rows per shared-memory stage

template <class T>
__global__ void __launch_bounds__(256)
k_gram_partial(int64_t n, int pa, int pb, const T* __restrict__ X, int64_t ldx,
               const T* __restrict__ Y, int64_t ldy, int ntb, bool hermitian,
               int64_t rows_per_split, T* __restrict__ part) {
  __shared__ T Xs[GRK][GT + 1];
  __shared__ T Ys[GRK][GT + 1];
  // decode the tile pair
  int ta, tb;
  const int pid = blockIdx.x;
  if (hermitian) {
    // enumerate pairs ta <= tb row by row
    int t = pid, a = 0;
    while (t >= ntb - a) { t -= ntb - a; ++a; }
    ta = a;
    tb = a + t;
  } else {
    ta = pid / ntb;
    tb = pid % ntb;
  }
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r1 = min(n, r0 + rows_per_split);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = szero<T>();

  for (int64_t rb = r0; rb < r1; rb += GRK) {
    for (int e = threadIdx.x; e < GRK * GT; e += 256) {
      const int r = e / GT, c = e % GT;
      const int64_t row = rb + r;
      const int ca = ta * GT + c, cb = tb * GT + c;
      Xs[r][c] = (row < r1 && ca < pa) ? X[row * ldx + ca] : szero<T>();
      Ys[r][c] = (row < r1 && cb < pb) ? Y[row * ldy + cb] : szero<T>();
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < GRK; ++r) {
      const T a0 = Xs[r][ty * 2], a1 = Xs[r][ty * 2 + 1];
      const T b0 = Ys[r][tx * 2], b1 = Ys[r][tx * 2 + 1];
      madd_conj(acc[0][0], a0, b0);
      madd_conj(acc[0][1], a0, b1);
      madd_conj(acc[1][0], a1, b0);
      madd_conj(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  T* P = part + (int64_t)blockIdx.y * pa * pb;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gi = ta * GT + ty * 2 + i, gj = tb * GT + tx * 2 + j;
      if (gi < pa && gj < pb) P[(int64_t)gi * pb + gj] = acc[i][j];
    }
}

template <class T>
__global__ void k_gram_reduce(int pa, int pb, int nsplit, bool hermitian, const T* __restrict__ part,
                              T* __restrict__ G, int64_t ldg) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)pa * pb) return;
  const int i = (int)(idx / pb), j = (int)(idx % pb);
  const bool mirror = hermitian && (i / GT > j / GT);
  const int si = mirror ? j : i, sj = mirror ? i : j;
  T s = szero<T>();
  for (int k = 0; k < nsplit; ++k) s = add(s, part[(int64_t)k * pa * pb + (int64_t)si * pb + sj]);
  G[(int64_t)i * ldg + j] = mirror ? conj_(s) : s;
}

template <class T>
void gram(apf_ctx* ctx, int64_t n, int64_t pa, int64_t pb, const T* X, int64_t ldx, const T* Y,
          int64_t ldy, T* G, int64_t ldg, bool hermitian) {
  if (pa == 0 || pb == 0) return;
  // hermitian: only tiles on and above the diagonal are computed; the others
  // are the conjugate transposes.  Exact for X == Y; for X != Y it is the
  // upper part of a product known to be Hermitian (X^H A X with A = A^H).
  APF_REQUIRE(!hermitian || pa == pb, APF_ERR_ARG);
  const int nta = (int)((pa + GT - 1) / GT), ntb = (int)((pb + GT - 1) / GT);
  const int npairs = hermitian ? nta * (nta + 1) / 2 : nta * ntb;
  int64_t nsplit = (4LL * ctx->num_sms + npairs - 1) / npairs;
  const int64_t max_split = (n + 255) / 256;
  if (nsplit > max_split) nsplit = max_split;
  if (nsplit < 1) nsplit = 1;
  int64_t rows = (n + nsplit - 1) / nsplit;
  rows = round_up(rows, GRK);
  nsplit = (n + rows - 1) / rows;
  if (nsplit < 1) nsplit = 1;
  DBuf part((size_t)nsplit * pa * pb * sizeof(T), ctx->stream, true);
  dim3 grid((unsigned)npairs, (unsigned)nsplit);
  k_gram_partial<T><<<grid, 256, 0, ctx->stream>>>(n, (int)pa, (int)pb, X, ldx, Y, ldy, ntb,
                                                  hermitian, rows, part.as<T>());
  const int64_t tot = pa * pb;
  k_gram_reduce<T><<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(
      (int)pa, (int)pb, (int)nsplit, hermitian, part.as<T>(), G, ldg);
  count_launch(ctx, 2);
}
template void gram<double>(apf_ctx*, int64_t, int64_t, int64_t, const double*, int64_t,
                           const double*, int64_t, double*, int64_t, bool);
template void gram<double2>(apf_ctx*, int64_t, int64_t, int64_t, const double2*, int64_t,
                            const double2*, int64_t, double2*, int64_t, bool);

// ---- Z = beta Z0 + alpha X M --------------------------------------------------
constexpr int MR = 64;  // rows per CTA
constexpr int MC = 32;  // columns per CTA
constexpr int MK = 16;  // k chunk

template <class T>
__global__ void __launch_bounds__(256)
k_gemm_tall(int64_t n, int pa, int pb, const T* __restrict__ X, int64_t ldx,
            const T* __restrict__ M, int64_t ldm, T* Z, int64_t ldz, double alpha, double beta,
            const T* Z0, int64_t ldz0, bool upper) {
  __shared__ T Xs[MR][MK + 1];
  __shared__ T Ms[MK][MC + 1];
  const int j0 = blockIdx.x * MC;
  const int64_t i0 = (int64_t)blockIdx.y * MR;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 2 columns x 4 rows per thread
  T acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = szero<T>();
  int kend = pa;
  if (upper && j0 + MC < kend) kend = j0 + MC;
  for (int k0 = 0; k0 < kend; k0 += MK) {
    for (int e = threadIdx.x; e < MR * MK; e += 256) {
      const int r = e / MK, c = e % MK;
      const int64_t row = i0 + r;
      Xs[r][c] = (row < n && k0 + c < pa) ? X[row * ldx + k0 + c] : szero<T>();
    }
    for (int e = threadIdx.x; e < MK * MC; e += 256) {
      const int r = e / MC, c = e % MC;
      Ms[r][c] = (k0 + r < pa && j0 + c < pb) ? M[(int64_t)(k0 + r) * ldm + j0 + c] : szero<T>();
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < MK; ++k) {
      const T m0 = Ms[k][tx * 2], m1 = Ms[k][tx * 2 + 1];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const T x = Xs[ty * 4 + i][k];
        madd(acc[i][0], x, m0);
        madd(acc[i][1], x, m1);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = i0 + ty * 4 + i;
    if (row >= n) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int col = j0 + tx * 2 + j;
      if (col >= pb) continue;
      T v = rmul(alpha, acc[i][j]);
      if (beta != 0.0) v = add(v, rmul(beta, Z0[row * ldz0 + col]));
      Z[row * ldz + col] = v;
    }
  }
}

template <class T>
void gemm_tall(apf_ctx* ctx, int64_t n, int64_t pa, int64_t pb, const T* X, int64_t ldx,
               const T* M, int64_t ldm, T* Z, int64_t ldz, double alpha, double beta, const T* Z0,
               int64_t ldz0, bool upper) {
  if (n == 0 || pb == 0) return;
  dim3 grid((unsigned)((pb + MC - 1) / MC), (unsigned)((n + MR - 1) / MR));
  k_gemm_tall<T><<<grid, 256, 0, ctx->stream>>>(n, (int)pa, (int)pb, X, ldx, M, ldm, Z, ldz,
                                                alpha, beta, Z0, ldz0, upper);
  count_launch(ctx);
}
template void gemm_tall<double>(apf_ctx*, int64_t, int64_t, int64_t, const double*, int64_t,
                                const double*, int64_t, double*, int64_t, double, double,
                                const double*, int64_t, bool);
template void gemm_tall<double2>(apf_ctx*, int64_t, int64_t, int64_t, const double2*, int64_t,
                                 const double2*, int64_t, double2*, int64_t, double, double,
                                 const double2*, int64_t, bool);

// ---- small C = alpha op(A) op(B) + beta C, one thread per output ---------------
template <class T>
__global__ void k_small_gemm(int m, int n, int k, bool ha, const T* __restrict__ A, int64_t lda,
                             bool hb, const T* __restrict__ B, int64_t ldb, T* C, int64_t ldc,
                             double alpha, double beta) {
  const int i = blockIdx.y * 16 + threadIdx.y;
  const int j = blockIdx.x * 16 + threadIdx.x;
  if (i >= m || j >= n) return;
  T s = szero<T>();
  for (int t = 0; t < k; ++t) {
    const T a = ha ? conj_(A[(int64_t)t * lda + i]) : A[(int64_t)i * lda + t];
    const T b = hb ? conj_(B[(int64_t)j * ldb + t]) : B[(int64_t)t * ldb + j];
    madd(s, a, b);
  }
  T v = rmul(alpha, s);
  if (beta != 0.0) v = add(v, rmul(beta, C[(int64_t)i * ldc + j]));
  C[(int64_t)i * ldc + j] = v;
}

template <class T>
void small_gemm(apf_ctx* ctx, int64_t m, int64_t n, int64_t k, char opa, const T* A, int64_t lda,
                char opb, const T* B, int64_t ldb, T* C, int64_t ldc, double alpha, double beta) {
  if (m == 0 || n == 0) return;
  dim3 block(16, 16), grid((unsigned)((n + 15) / 16), (unsigned)((m + 15) / 16));
  k_small_gemm<T><<<grid, block, 0, ctx->stream>>>((int)m, (int)n, (int)k, opa == 'H', A, lda,
                                                   opb == 'H', B, ldb, C, ldc, alpha, beta);
  count_launch(ctx);
}
template void small_gemm<double>(apf_ctx*, int64_t, int64_t, int64_t, char, const double*, int64_t,
                                 char, const double*, int64_t, double*, int64_t, double, double);
template void small_gemm<double2>(apf_ctx*, int64_t, int64_t, int64_t, char, const double2*,
                                  int64_t, char, const double2*, int64_t, double2*, int64_t,
                                  double, double);

}  // namespace apf

namespace apf {

// G = X^H Y like gram() (full, non-Hermitian tiling), with the split partials
// in caller-provided device scratch instead of an allocation: the number of
// row splits is capped so that nsplit * pa * pb elements fit scratch_bytes.
// Every partial entry that the reduction reads is written first, so the
// scratch needs no clearing.  Launches on `stream`; throws ApfError.
template <class T>
void gram_scratch(cudaStream_t stream, int num_sms, int64_t n, int64_t pa, int64_t pb, const T* X,
                  int64_t ldx, const T* Y, int64_t ldy, T* G, int64_t ldg, void* scratch,
                  size_t scratch_bytes) {
  const size_t per_split = (size_t)pa * pb * sizeof(T);
  APF_REQUIRE(per_split <= scratch_bytes, APF_ERR_ARG);
  const int nta = (int)((pa + GT - 1) / GT), ntb = (int)((pb + GT - 1) / GT);
  const int npairs = nta * ntb;
  int64_t nsplit = (4LL * num_sms + npairs - 1) / npairs;
  const int64_t max_split = (n + 255) / 256;
  if (nsplit > max_split) nsplit = max_split;
  const int64_t cap = (int64_t)(scratch_bytes / per_split);
  if (nsplit > cap) nsplit = cap;
  if (nsplit < 1) nsplit = 1;
  int64_t rows = (n + nsplit - 1) / nsplit;
  rows = round_up(rows, GRK);
  nsplit = (n + rows - 1) / rows;
  if (nsplit < 1) nsplit = 1;
  T* part = static_cast<T*>(scratch);
  dim3 grid((unsigned)npairs, (unsigned)nsplit);
  k_gram_partial<T><<<grid, 256, 0, stream>>>(n, (int)pa, (int)pb, X, ldx, Y, ldy, ntb, false, rows, part);
  const int64_t tot = pa * pb;
  k_gram_reduce<T><<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>((int)pa, (int)pb, (int)nsplit, false,
                                                                    part, G, ldg);
  APF_CUDA(cudaGetLastError());
}
template void gram_scratch<double>(cudaStream_t, int, int64_t, int64_t, int64_t, const double*, int64_t,
                                   const double*, int64_t, double*, int64_t, void*, size_t);
template void gram_scratch<double2>(cudaStream_t, int, int64_t, int64_t, int64_t, const double2*, int64_t,
                                    const double2*, int64_t, double2*, int64_t, void*, size_t);

}  // namespace apf
