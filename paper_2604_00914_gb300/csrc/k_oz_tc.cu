// FP64-accurate dense products on the tcgen05 tensor cores: the Gram matrices
// X^H Y of the Cholesky QR and Rayleigh-Ritz steps of Alg. 4, and the tall
// block products Z = beta Z0 + alpha X M that apply their small factors.
//
// Method (the Ozaki scheme: Ozaki, Ogita, Oishi and Rump, Numer. Algorithms
// 59, 2012; integer slices as in Ootomo, Ozaki and Yokota, IJHPCA 2024).
// Every product is written as a real "NT" product C[m][n] = sum_k A[m][k] B[n][k]
// (a complex product becomes a real one of twice the length: the real and
// imaginary parts are stacked along k, see gram_tc and gemm_tall_tc).  Each
// row m of A (each row n of B) has an exponent E with |entries| < 2^E; the
// integer F = round(x 2^(55 - E)) (|F| < 2^55) is cut into seven balanced
// base-256 digits sigma_0..sigma_6 in [-128, 128], F = sum_s sigma_s 2^(8 (6 - s)),
// held exactly in bf16.  Then
//     C[m][n] ~ 2^(E_m + F_n - 62) sum_{d=0}^{6} 2^(8 (6 - d)) P_d,
//     P_d = sum_{s + t = d} sum_k sigma_s(A)[m][k] sigma_t(B)[n][k],
// dropping the pairs s + t >= 7 (below 2^-56 of the leading term, as the
// rounding of F).  P_d gains at most (d + 1) x 32 x 2^14 in magnitude per
// 32-wide chunk of k, so the tensor cores' FP32 accumulation stays exact (every
// partial sum an integer within 2^24) over floor(32 / (d + 1)) chunks: from 32
// chunks for d = 0 to 4 for d = 6.  At the end of each such period the FP32 sum
// is read out, converted to an integer exactly, and added into two 64-bit
// integers per output element,
//     hi = P_0 2^16 + P_1 2^8 + P_2,  lo = P_3 2^24 + P_4 2^16 + P_5 2^8 + P_6,
// so C = 2^(E_m + F_n - 62) (hi 2^32 + lo) is formed once, in FP64.  (FP64
// arithmetic runs at a tiny fraction of the tensor rate on this part: the
// carry never touches it.)  Split-K partial sums are added with 64-bit
// integer atomics, which is exact and independent of the order.
//
// Kernel (one CTA per 128 x nt output tile, nt <= 64, and K range; 320
// threads, details at k_oz_umma): a producer warp brings the digit tiles of
// each chunk into a two-stage ring with bulk copies (cp.async.bulk) of
// pre-swizzled (64-byte swizzle) digit planes, one mbarrier per digit; an MMA
// warp issues the 28 digit pairs of a chunk (2 k steps each) as tcgen05.mma
// (M = 128, N = nt, K = 16, bf16 in, FP32 accumulate) into seven TMEM
// accumulators of 64 columns, one per diagonal; eight drain warps read an
// accumulator with tcgen05.ld when its period ends.  The MMA reads A (128 x 16)
// and B (nt x 16) from shared memory for 2 x 128 x nt x 16 flops: a 64-wide
// tile reads 40 % fewer operand bytes per flop than a 32-wide one.
// Every wait is bounded in time and a timeout makes all roles stop, let their
// copies and MMAs in flight complete, free the TMEM and record
// DEV_BARRIER_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>

#include "apf_internal.h"
#include "spmm_sell.cuh"

namespace apf {

constexpr int OZS = 7;        // digits per value
constexpr int OZ_BM = 128;    // output tile rows (MMA M)
constexpr int OZ_BN = 64;     // output tile columns (MMA N; the last tile of a range may be narrower)
constexpr int OZ_NQ = 16;     // granularity of a tile's width (MMA N multiple of 16 for M = 128)
constexpr int OZ_KC = 32;     // k per chunk (one 64-byte swizzle row of bf16)
constexpr uint32_t OZ_A_SLICE = OZ_BM * OZ_KC * 2;   // 8 KB
constexpr uint32_t OZ_B_SLICE = OZ_BN * OZ_KC * 2;   // 4 KB (a narrower tile uses the front)
constexpr uint32_t OZ_A_STAGE = OZS * OZ_A_SLICE;    // 56 KB
constexpr uint32_t OZ_B_STAGE = OZS * OZ_B_SLICE;    // 28 KB
constexpr int OZ_STAGES = 2;                        // operand ring depth
constexpr size_t OZ_SMEM = 1024 + OZ_STAGES * (size_t)(OZ_A_STAGE + OZ_B_STAGE) + 1024;

// Drain period of diagonal d, in chunks: P_d gains at most (d + 1) x 32 x 2^14
// = (d + 1) 2^19 in magnitude per chunk, so floor(32 / (d + 1)) chunks keep
// every partial sum within 2^24, where FP32 holds integers exactly.
__host__ __device__ constexpr int oz_period(int d) { return 32 / (d + 1); }

// Digit layout in global memory: chunk-major planes S[kc][s][row][32 k], each
// 64-byte row already in the 64-byte-swizzled order the MMA reads from shared
// memory (16-byte unit u of row r stored at u ^ ((r >> 1) & 3)), so one
// contiguous bulk copy brings a slice's 128-row (or 32-row) tile of a chunk
// into its shared-memory image.
__device__ __forceinline__ int64_t oz_off(int64_t kc, int s, int64_t row, int64_t rowsP, int kk) {
  return ((kc * OZS + s) * rowsP + row) * OZ_KC + ((((kk >> 3) ^ (int)((row >> 1) & 3)) << 3) | (kk & 7));
}

// ---- digits ----------------------------------------------------------------
__device__ __forceinline__ double oz_abs_max(double v) { return fabs(v); }
__device__ __forceinline__ double oz_abs_max(double2 v) { return fmax(fabs(v.x), fabs(v.y)); }

// E with |v| < 2^E for v = the largest magnitude (0 for v = 0), from the bits
__device__ __forceinline__ int oz_exponent(double m) {
  const long long b = __double_as_longlong(m);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return m > 0.0 ? -1022 : 0;  // subnormal maxima: treat as 2^-1022
  return ex - 1022;                         // m = 1.f 2^(ex - 1023) < 2^(ex - 1022)
}

// balanced base-256 digits of round(x 2^(55 - E)), |x| < 2^E, by integer
// operations on the bits of x (no FP64 arithmetic)
__device__ __forceinline__ void oz_digits(double x, int E, int (&dg)[OZS]) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  long long F = 0;
  if (ex != 0) {
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
    const int sh = ex - 1020 - E;  // x = m 2^(ex - 1075): F = m 2^(ex - 1075 + 55 - E)
    if (sh >= 0) F = m << (sh > 2 ? 2 : sh);
    else if (sh > -62) F = (m + (1LL << (-sh - 1))) >> (-sh);
  }
  if (b < 0) F = -F;
#pragma unroll
  for (int s = OZS - 1; s >= 1; --s) {
    int d = (int)(F & 0xFF);
    if (d >= 128) d -= 256;
    dg[s] = d;
    F = (F - d) >> 8;
  }
  dg[0] = (int)F;
}

// v 2^e for |e| <= 2044 by two exact power-of-two multiplies (no library call)
__device__ __forceinline__ double oz_scale(double v, int e) {
  const int e1 = e / 2, e2 = e - e1;
  return v * __longlong_as_double((long long)(1023 + e1) << 52) * __longlong_as_double((long long)(1023 + e2) << 52);
}

__device__ __forceinline__ __nv_bfloat16 oz_bf16(int v) { return __float2bfloat16_rn((float)v); }

// per-column exponents of X (n x p, ld): part[block][c] maxima, then E
template <class T>
__global__ void k_ozt_colmax(int64_t n, int p, const T* __restrict__ X, int64_t ld, int64_t rows,
                             double* __restrict__ part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows, r1 = min(n, r0 + rows);
  double m = 0.0;
  for (int64_t i = r0; i < r1; ++i) m = fmax(m, oz_abs_max(X[i * ld + c]));
  part[(int64_t)blockIdx.y * p + c] = m;
}

__global__ void k_ozt_colexp(int p, int nb, const double* __restrict__ part, int* __restrict__ e, int pP) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= pP) return;
  double m = 0.0;
  if (c < p)
    for (int b = 0; b < nb; ++b) m = fmax(m, part[(int64_t)b * p + c]);
  e[c] = oz_exponent(m);
}

// Column digits, transposed: S[s][a][k] (k contiguous, KT per row), with
// k = i for the real part of row i and k = nK + i for the imaginary part.
template <class T, int C>
__global__ void __launch_bounds__(256)
k_ozt_split_cols(int64_t n, int p, const T* __restrict__ X, int64_t ld, const int* __restrict__ e, int64_t nK,
                 int64_t KT, int pP, __nv_bfloat16* __restrict__ S) {
  __shared__ __nv_bfloat16 tile[OZS][C][32][34];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int a0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r;
    const int a = a0 + tx;
    double part[2] = {0.0, 0.0};
    if (i < n && a < p) {
      const T v = X[i * ld + a];
      if constexpr (C == 2) {
        part[0] = reinterpret_cast<const double2&>(v).x;
        part[1] = reinterpret_cast<const double2&>(v).y;
      } else {
        part[0] = reinterpret_cast<const double&>(v);
      }
    }
    const int E = (a < pP) ? e[a] : 0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      int dg[OZS];
      oz_digits(part[c], E, dg);
#pragma unroll
      for (int s = 0; s < OZS; ++s) tile[s][c][tx][r] = oz_bf16(dg[s]);
    }
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {  // r: column within the tile, tx: row
    const int a = a0 + r;
    const int64_t i = i0 + tx;
    if (a >= pP || i >= nK) continue;
#pragma unroll
    for (int s = 0; s < OZS; ++s)
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int64_t k = (int64_t)c * nK + i;
        S[oz_off(k / OZ_KC, s, a, pP, (int)(k % OZ_KC))] = tile[s][c][r][tx];
      }
  }
}

// Row digits: S[s][i][k] for the stacked row (re_0..re_{p-1}, im_0..im_{p-1})
// of X (KT >= C p, zero beyond), exponent per row.
template <class T, int C>
__global__ void __launch_bounds__(256)
k_ozt_rowexp(int64_t n, int p, const T* __restrict__ X, int64_t ld, int64_t nP, int* __restrict__ e) {
  const int64_t i = (int64_t)blockIdx.x * 8 + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (i >= nP) return;
  double m = 0.0;
  if (i < n)
    for (int c = lane; c < p; c += 32) m = fmax(m, oz_abs_max(X[i * ld + c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) e[i] = oz_exponent(m);
}

template <class T, int C>
__global__ void __launch_bounds__(256)
k_ozt_split_rows(int64_t n, int p, const T* __restrict__ X, int64_t ld, const int* __restrict__ e, int64_t nP,
                 int64_t KT, __nv_bfloat16* __restrict__ S) {
  const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (idx >= nP * KT) return;
  const int64_t i = idx / KT;
  const int k = (int)(idx % KT);
  double x = 0.0;
  if (i < n && k < C * p) {
    const int c = k / p, col = k % p;
    const T v = X[i * ld + col];
    if constexpr (C == 2) x = c == 0 ? reinterpret_cast<const double2&>(v).x : reinterpret_cast<const double2&>(v).y;
    else x = reinterpret_cast<const double&>(v);
  }
  int dg[OZS];
  oz_digits(x, e[i], dg);
#pragma unroll
  for (int s = 0; s < OZS; ++s) S[oz_off(k / OZ_KC, s, i, nP, k % OZ_KC)] = oz_bf16(dg[s]);
}

// The real form of a small factor M (pa x pb, ldm): Bt[j][k] = Mt[k][j] with
// Mt = M (real) or [[Mr, Mi], [-Mi, Mr]] (complex; rows k < pa go with the real
// parts of X's row, k >= pa with the imaginary parts), then column digits of
// Mt: one block per output column j.
template <class T, int C>
__global__ void __launch_bounds__(256)
k_ozt_split_small(int pa, int pb, const T* __restrict__ M, int64_t ldm, int NP, int64_t KT,
                  __nv_bfloat16* __restrict__ S, int* __restrict__ f) {
  const int j = blockIdx.x;
  __shared__ double red[8];
  __shared__ int Esh;
  auto value = [&](int k) -> double {
    if (j >= C * pb || k >= C * pa) return 0.0;
    if constexpr (C == 1) {
      return reinterpret_cast<const double*>(M)[(int64_t)k * ldm + j];
    } else {
      const int jr = j % pb, part = j / pb;    // output column: real (0) or imaginary (1) part
      const int kr = k % pa, kpart = k / pa;   // row of M, and whether it multiplies re or im of X
      const double2 v = reinterpret_cast<const double2*>(M)[(int64_t)kr * ldm + jr];
      // Zr = Xr Mr - Xi Mi,  Zi = Xr Mi + Xi Mr
      if (part == 0) return kpart == 0 ? v.x : -v.y;
      return kpart == 0 ? v.y : v.x;
    }
  };
  double m = 0.0;
  for (int k = threadIdx.x; k < KT; k += 256) m = fmax(m, fabs(value(k)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < 8; ++w) mm = fmax(mm, red[w]);
    Esh = oz_exponent(mm);
    f[j] = Esh;
  }
  __syncthreads();
  const int E = Esh;
  for (int k = threadIdx.x; k < KT; k += 256) {
    int dg[OZS];
    oz_digits(value(k), E, dg);
#pragma unroll
    for (int s = 0; s < OZS; ++s) S[oz_off(k / OZ_KC, s, j, NP, (int)(k % OZ_KC))] = oz_bf16(dg[s]);
  }
}

// ---- tcgen05 primitives ---------------------------------------------------------
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(holder)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// D = A B^T (the first product of an accumulation) and D += A B^T
__device__ __forceinline__ void umma_bf16_first(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 0, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc)
      : "memory");
}
__device__ __forceinline__ void umma_bf16_acc(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.eq.b32 p, 0, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 64-byte swizzle (8-row atoms of
// 512 bytes, stacked 512 bytes apart), tcgen05 descriptor version 1
__device__ __forceinline__ uint64_t umma_desc_sw64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(512 >> 4) << 32;     // stride byte offset
  d |= (uint64_t)1 << 46;              // version
  d |= (uint64_t)4 << 61;              // SWIZZLE_64B
  return d;
}
// instruction descriptor: D FP32, A and B bf16, both K-major, M x N, B negated on request
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N, bool neg_b) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((neg_b ? 1u : 0u) << 14) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// the first `lanes` threads of the calling warp wait for a barrier phase; all
// roles give up when the shared abort flag is set
__device__ __forceinline__ bool oz_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = sell_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (sell_ns() - t0 > limit_ns) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

struct OzTile {
  int m0, n0, nt, pad;  // first output row and column, width (a multiple of 16, <= 64)
};

struct OzArgs {
  const __nv_bfloat16* SA;  // digit planes of A (rowsA rows) and B (rowsB rows)
  const __nv_bfloat16* SB;
  int64_t rowsA, rowsB;
  int mode;          // 0: Gram (int64 atomics into H, L); 1: tall product (FP64 out)
  int64_t chunks;    // k chunks of this product (KT / OZ_KC)
  int64_t chunks_per_split;
  const OzTile* tiles;  // per blockIdx.x
  // mode 0: complex Im half of the n range: B rows shifted by half_k chunks, negated past it
  int n_im0;         // first n of the imaginary half (or a large value)
  int64_t half_chunks;
  unsigned long long* H;  // [MP][NP]
  unsigned long long* L;
  int NP;
  // mode 1
  int64_t nrows;     // rows of Z
  int ncols;         // real columns (C pb)
  int pb;            // complex: columns of Z; real: = ncols
  int cplx;
  const int* ea;     // row exponents of A
  const int* fb;     // row exponents of B
  double* Z;         // FP64 (re, im interleaved for complex)
  const double* Z0;
  int64_t ldz, ldz0; // in complex elements for complex
  double alpha, beta;
  int* err;
  uint64_t limit_ns;
};

constexpr int OZ_THREADS = 320;
constexpr int OZ_DRAIN = 256;       // drain threads (warps 0-7)

// One CTA: a 128 x nt output tile over one range of k chunks.
//   warp 8 (lane 0)  producer: per chunk and digit s, one bulk copy of the A
//                    tile (128 rows x 32 k) and one of the B tile (nt rows),
//                    completing on the barrier of (stage, s), so the MMAs of
//                    diagonal d start once digits 0..d have landed;
//   warp 9 (lane 0)  MMA issuer: diagonal d of a chunk is the d + 1 digit
//                    pairs (s, d - s), two k steps each, accumulated into TMEM
//                    columns 64 d .. 64 d + nt - 1; the first product of a
//                    drain period overwrites;
//   warps 0-7        drain: at the end of each period of diagonal d (and of
//                    the range) read its accumulator (warp w: TMEM lanes
//                    32 (w mod 4) .., columns 32 (w / 4) ..), convert the exact
//                    FP32 integers and add them, shifted by the diagonal's
//                    weight, into two 64-bit integers per output element:
//                    hi = P_0 2^16 + P_1 2^8 + P_2, lo = P_3 2^24 + ... + P_6.
__global__ void __launch_bounds__(OZ_THREADS, 1)
k_oz_umma(OzArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1 KB-aligned operand area (the swizzle atoms need 512-byte alignment)
  const uint32_t base_s = smem_addr(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (base_s & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);        // [stage][digit] bulk copies -> MMA
  uint64_t* empty = full + OZ_STAGES * OZS;                   // [stage] MMA -> producer
  uint64_t* tfull = empty + OZ_STAGES;                        // [d] MMA -> drain
  uint64_t* tempty = tfull + OZS;                             // [d] drain -> MMA
  uint64_t* fin = tempty + OZS;                               // MMAs in flight at an abort
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  int* issued = const_cast<int*>(abort_flag) + 1;             // chunks the producer issued
  int* fin_armed = issued + 1;                                // the MMA issuer committed `fin`
  unsigned char* opA = smem + 1024;
  unsigned char* opB = opA + OZ_STAGES * OZ_A_STAGE;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const OzTile tile = a.tiles[blockIdx.x];
  const int m0 = tile.m0, n0 = tile.n0, nt = tile.nt;
  const int64_t c_begin = (int64_t)blockIdx.y * a.chunks_per_split;
  const int64_t c_end = min(a.chunks, c_begin + a.chunks_per_split);
  const int nch = (int)(c_end > c_begin ? c_end - c_begin : 0);

  if (threadIdx.x == 0) {
    for (int i = 0; i < OZ_STAGES * OZS; ++i) mbar_init(full + i, 1);
    for (int i = 0; i < OZ_STAGES; ++i) mbar_init(empty + i, 1);
    for (int d = 0; d < OZS; ++d) {
      mbar_init(tfull + d, 1);
      mbar_init(tempty + d, OZ_DRAIN);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    *issued = 0;
    *fin_armed = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_holder, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tmem_holder;

  // the imaginary half of a complex Gram: B rows from the other half of k, negated in the second
  const bool im_tile = a.mode == 0 && n0 >= a.n_im0;
  const uint32_t b_bytes = (uint32_t)nt * OZ_KC * 2;

  if (warp == 8) {
    if (lane == 0) {
      const int nb = im_tile ? n0 - a.n_im0 : n0;
      int c = 0;
      for (; c < nch; ++c) {
        const int st = c % OZ_STAGES, use = c / OZ_STAGES;
        if (c >= OZ_STAGES && !oz_wait(empty + st, (uint32_t)((use - 1) & 1), a.limit_ns, abort_flag)) break;
        const int64_t kc = c_begin + c;
        int64_t kb = kc;
        if (im_tile) kb = kc < a.half_chunks ? kc + a.half_chunks : kc - a.half_chunks;
        for (int sl = 0; sl < OZS; ++sl) {
          uint64_t* bar = full + st * OZS + sl;
          mbar_arrive_expect(bar, OZ_A_SLICE + b_bytes);
          bulk_g2s(opA + st * OZ_A_STAGE + sl * OZ_A_SLICE, a.SA + oz_off(kc, sl, m0, a.rowsA, 0), OZ_A_SLICE, bar);
          bulk_g2s(opB + st * OZ_B_STAGE + sl * OZ_B_SLICE, a.SB + oz_off(kb, sl, nb, a.rowsB, 0), b_bytes, bar);
        }
      }
      *issued = c;
    }
  } else if (warp == 9) {
    if (lane == 0) {
      const uint32_t id_pos = umma_idesc(OZ_BM, nt, false);
      const uint32_t id_neg = umma_idesc(OZ_BM, nt, true);
      bool any = false;
      for (int c = 0; c < nch && !*abort_flag; ++c) {
        const int st = c % OZ_STAGES;
        const uint32_t ph = (uint32_t)((c / OZ_STAGES) & 1);
        const uint32_t idesc = (im_tile && c_begin + c >= a.half_chunks) ? id_neg : id_pos;
        // descriptors of the stage's first tiles; the other tiles are at fixed
        // offsets (the 14-bit address field holds addr / 16 and never carries)
        const uint64_t ad0 = umma_desc_sw64(smem_addr(opA + st * OZ_A_STAGE));
        const uint64_t bd0 = umma_desc_sw64(smem_addr(opB + st * OZ_B_STAGE));
        bool ok = true;
#pragma unroll
        for (int d = 0; d < OZS; ++d) {
          const int per = oz_period(d);
          const bool first = c % per == 0;
          if (!oz_wait(full + st * OZS + d, ph, a.limit_ns, abort_flag)) { ok = false; break; }
          if (first && c > 0 &&
              !oz_wait(tempty + d, (uint32_t)((c / per - 1) & 1), a.limit_ns, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dt = tbase + (uint32_t)(d * OZ_BN);
#pragma unroll
          for (int s = 0; s <= d; ++s) {
#pragma unroll
            for (int kk = 0; kk < OZ_KC / 16; ++kk) {
              const uint64_t ad = ad0 + (uint64_t)((s * OZ_A_SLICE + kk * 32) >> 4);
              const uint64_t bd = bd0 + (uint64_t)(((d - s) * OZ_B_SLICE + kk * 32) >> 4);
              if (first && s == 0 && kk == 0) umma_bf16_first(dt, ad, bd, idesc);
              else umma_bf16_acc(dt, ad, bd, idesc);
            }
          }
          any = true;
          if ((c + 1) % per == 0 || c == nch - 1) umma_commit(tfull + d);
        }
        if (!ok) break;
        umma_commit(empty + st);
      }
      if (*abort_flag && any) {
        umma_commit(fin);
        *fin_armed = 1;
      }
    }
  } else {
    const int quarter = warp & 3, half = warp >> 2;
    const int col0 = half * 32;            // first column of this warp within the tile
    const bool active = col0 < nt;
    const bool second = nt - col0 > 16;    // its second group of 16 columns is in the tile
    long long hi[32], lo[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    bool ok = true;
    for (int c = 0; c < nch && ok; ++c) {
#pragma unroll
      for (int d = 0; d < OZS; ++d) {
        const int per = oz_period(d);
        if (!((c + 1) % per == 0 || c == nch - 1)) continue;
        if (!oz_wait(tfull + d, (uint32_t)((c / per) & 1), a.limit_ns, abort_flag)) { ok = false; break; }
        tc_fence_after();
        // weights: hi = P0 2^16 + P1 2^8 + P2, lo = P3 2^24 + P4 2^16 + P5 2^8 + P6
        constexpr int kShift[OZS] = {16, 8, 0, 24, 16, 8, 0};
        uint32_t r[16];
        if (active) {
          tmem_ld16(tbase + lane_off + (uint32_t)(d * OZ_BN + col0), r);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const long long v = (long long)__float2int_rn(__uint_as_float(r[j])) << kShift[d];
            if (d < 3) hi[j] += v;
            else lo[j] += v;
          }
          if (second) {
            tmem_ld16(tbase + lane_off + (uint32_t)(d * OZ_BN + col0 + 16), r);
            tmem_wait_ld();
          }
        }
        tc_fence_before();
        mbar_arrive(tempty + d);
        if (active && second) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const long long v = (long long)__float2int_rn(__uint_as_float(r[j])) << kShift[d];
            if (d < 3) hi[16 + j] += v;
            else lo[16 + j] += v;
          }
        }
      }
    }
    if (ok && !*abort_flag && active) {
      const int m = m0 + quarter * 32 + lane;
      const int cend = min(nt - col0, 32);
      if (a.mode == 0) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (j >= cend) break;
          const int64_t o = (int64_t)m * a.NP + n0 + col0 + j;
          if (hi[j]) atomicAdd(a.H + o, (unsigned long long)hi[j]);
          if (lo[j]) atomicAdd(a.L + o, (unsigned long long)lo[j]);
        }
      } else if (m < a.nrows) {
        const int em = a.ea[m];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + col0 + j;
          if (j >= cend || col >= a.ncols) break;
          const int sc = em + a.fb[col] - 62;
          const double v = oz_scale((double)hi[j], sc + 32) + oz_scale((double)lo[j], sc);
          int64_t oz, oz0;
          if (a.cplx) {
            const int jc = col % a.pb, part = col / a.pb;
            oz = (m * a.ldz + jc) * 2 + part;
            oz0 = (m * a.ldz0 + jc) * 2 + part;
          } else {
            oz = m * a.ldz + col;
            oz0 = m * a.ldz0 + col;
          }
          const double z0 = a.beta != 0.0 ? a.beta * a.Z0[oz0] : 0.0;
          a.Z[oz] = fma(a.alpha, v, z0);
        }
      }
    }
  }
  // every role is done (or gave up): wait for copies and MMAs still in flight
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) atomicCAS(a.err, 0, DEV_BARRIER_TIMEOUT);
    volatile int dummy = 0;
    if (warp == 8 && lane == 0) {
      // the last chunks' bulk copies complete by themselves: wait for them
      // (bounded) before the shared memory goes away
      const int n_is = *issued;
      for (int c = (n_is > OZ_STAGES ? n_is - OZ_STAGES : 0); c < n_is; ++c)
        for (int sl = 0; sl < OZS; ++sl)
          oz_wait(full + (c % OZ_STAGES) * OZS + sl, (uint32_t)((c / OZ_STAGES) & 1), 1000000000ull, &dummy);
    }
    if (warp == 9 && lane == 0 && *fin_armed)
      oz_wait(fin, 0u, 1000000000ull, &dummy);  // every MMA issued has completed
    __syncthreads();
  }
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

// hi/lo sums of the Gram -> G (FP64), mirroring the tiles below the diagonal
// last column of the output tile that holds column j of a range of pbP columns
__host__ __device__ inline int oz_tile_end(int j, int pbP) {
  const int b0 = (j / OZ_BN) * OZ_BN;
  return (b0 + OZ_BN < pbP ? b0 + OZ_BN : pbP) - 1;
}

template <class T>
__global__ void k_oz_gram_finish(int pa, int pb, int pbP, int NP, int n_im0, bool hermitian,
                                 const unsigned long long* __restrict__ H, const unsigned long long* __restrict__ L,
                                 const int* __restrict__ ea, const int* __restrict__ eb, T* __restrict__ G,
                                 int64_t ldg) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)pa * pb) return;
  const int i = (int)(idx / pb), j = (int)(idx % pb);
  // computed tiles: (tile m, tile n) with n range reaching the m range's start
  const bool have = !hermitian || oz_tile_end(j, pbP) >= (i / OZ_BM) * OZ_BM;
  const int si = have ? i : j, sj = have ? j : i;
  auto val = [&](int col) {
    const int64_t o = (int64_t)si * NP + col;
    const int sc = ea[si] + eb[sj] - 62;
    return oz_scale((double)(long long)H[o], sc + 32) + oz_scale((double)(long long)L[o], sc);
  };
  const double re = val(sj);
  if constexpr (ScalarTraits<T>::is_complex) {
    const double im = val(n_im0 + sj);
    G[(int64_t)i * ldg + j] = make_double2(re, have ? im : -im);
  } else {
    G[(int64_t)i * ldg + j] = re;
  }
}

// ---- host ----------------------------------------------------------------------
// Context workspace: grown on demand in stream order, kept until apf_destroy.
static void* workspace(apf_ctx* ctx, size_t bytes) {
  if (ctx->ws_bytes < bytes) {
    if (ctx->ws) APF_CUDA(cudaFreeAsync(ctx->ws, ctx->stream));
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    const size_t grow = bytes + bytes / 4;
    APF_CUDA(cudaMallocAsync(&ctx->ws, grow, ctx->stream));
    ctx->ws_bytes = grow;
  }
  return ctx->ws;
}

static void launch_oz(apf_ctx* ctx, OzArgs& a, int ntiles, int nsplit) {
  allow_large_smem_bytes<k_oz_umma>(ctx->device, (int)OZ_SMEM);
  a.err = ctx->d_err;
  a.limit_ns = filter_wait_ns(ctx);
  k_oz_umma<<<dim3((unsigned)ntiles, (unsigned)nsplit), OZ_THREADS, OZ_SMEM, ctx->stream>>>(a);
  count_launch(ctx);
}

// Output tiles of width <= OZ_BN (multiples of OZ_NQ) over columns [c0, c0 + w).
static void push_tiles(std::vector<OzTile>& t, int m0, int c0, int w) {
  for (int b = 0; b < w; b += OZ_BN) t.push_back(OzTile{m0, c0 + b, std::min(OZ_BN, w - b), 0});
}

// K splits per tile: one CTA per SM at a time, so pick the split count whose
// grid fills whole waves best (one to four waves), keeping >= 8 chunks a CTA.
static int64_t pick_splits(int ntiles, int64_t chunks, int num_sms) {
  const int64_t cap = std::max<int64_t>(1, chunks / 8);
  if (ntiles >= num_sms) return 1;
  int64_t best = 1;
  double best_eff = -1.0;
  for (int w = 1; w <= 4; ++w) {
    const int64_t ns = std::min<int64_t>(cap, std::max<int64_t>(1, (int64_t)w * num_sms / ntiles));
    const int64_t total = ns * ntiles;
    const double eff = (double)total / (double)(((total + num_sms - 1) / num_sms) * num_sms);
    if (eff > best_eff + 1e-9) { best_eff = eff; best = ns; }
  }
  return best;
}

template <class T>
void gram_tc(apf_ctx* ctx, int64_t n, int64_t pa, int64_t pb, const T* X, int64_t ldx, const T* Y, int64_t ldy,
             T* G, int64_t ldg, bool hermitian) {
  if (pa == 0 || pb == 0) return;
  APF_REQUIRE(!hermitian || pa == pb, APF_ERR_ARG);
  APF_REQUIRE(n >= 1 && pa <= APF_MAX_P && pb <= APF_MAX_P, APF_ERR_ARG);
  constexpr int C = ScalarTraits<T>::is_complex ? 2 : 1;
  const int64_t nK = round_up(n, OZ_KC), KT = C * nK;
  // exactness of the carry: at most 2^16 chunks of k in all
  if (KT / OZ_KC > 65536) { gram<T>(ctx, n, pa, pb, X, ldx, Y, ldy, G, ldg, hermitian); return; }
  const int paP = (int)round_up(pa, OZ_BM), pbP = (int)round_up(pb, OZ_NQ);
  const int NP = C * pbP;  // output columns: [re | im]
  const bool same = (X == Y && ldx == ldy && pa == pb);
  const int pyP = same ? paP : pbP;  // rows of Y's slice array
  // workspace: slices of X and Y, exponents, hi/lo sums, tile list, column maxima
  const int64_t nb = std::min<int64_t>(std::max<int64_t>(1, 4LL * ctx->num_sms), n);
  const int64_t rows_per = (n + nb - 1) / nb;
  const size_t sx = (size_t)OZS * paP * KT * 2, sy = same ? 0 : (size_t)OZS * pyP * KT * 2;
  const size_t hl = (size_t)paP * NP * 8;
  const int ntm = paP / OZ_BM;
  std::vector<OzTile> tiles;
  for (int tm = 0; tm < ntm; ++tm)
    for (int part = 0; part < C; ++part) {
      std::vector<OzTile> row;
      push_tiles(row, tm * OZ_BM, 0, pbP);
      for (const OzTile& t : row) {
        // below the diagonal of a Hermitian Gram: mirrored by the finish kernel
        if (hermitian && oz_tile_end(t.n0, pbP) < tm * OZ_BM) continue;
        tiles.push_back(OzTile{t.m0, t.n0 + part * pbP, t.nt, 0});
      }
    }
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off = round_up((int64_t)(off + b), 1024); return o; };
  const size_t o_sx = take(sx), o_sy = take(sy), o_ex = take((size_t)paP * 4), o_ey = take((size_t)pyP * 4);
  const size_t o_h = take(hl), o_l = take(hl), o_t = take(tiles.size() * sizeof(OzTile));
  const size_t o_part = take((size_t)nb * std::max(pa, pb) * 8);
  unsigned char* ws = static_cast<unsigned char*>(workspace(ctx, off));
  auto* SX = reinterpret_cast<__nv_bfloat16*>(ws + o_sx);
  auto* SY = same ? SX : reinterpret_cast<__nv_bfloat16*>(ws + o_sy);
  int* ex = reinterpret_cast<int*>(ws + o_ex);
  int* ey = same ? ex : reinterpret_cast<int*>(ws + o_ey);
  auto* H = reinterpret_cast<unsigned long long*>(ws + o_h);
  auto* L = reinterpret_cast<unsigned long long*>(ws + o_l);
  OzTile* dtiles = reinterpret_cast<OzTile*>(ws + o_t);
  double* part = reinterpret_cast<double*>(ws + o_part);
  APF_CUDA(cudaMemcpyAsync(dtiles, tiles.data(), tiles.size() * sizeof(OzTile), cudaMemcpyHostToDevice,
                           ctx->stream));
  APF_CUDA(cudaMemsetAsync(H, 0, 2 * hl + (o_l - o_h - hl), ctx->stream));

  auto slice = [&](const T* M, int64_t ld, int64_t p, int pP, int* e, __nv_bfloat16* S) {
    k_ozt_colmax<T><<<dim3((unsigned)((p + 127) / 128), (unsigned)nb), 128, 0, ctx->stream>>>(n, (int)p, M, ld,
                                                                                           rows_per, part);
    k_ozt_colexp<<<(unsigned)((pP + 127) / 128), 128, 0, ctx->stream>>>((int)p, (int)nb, part, e, pP);
    k_ozt_split_cols<T, C><<<dim3((unsigned)(nK / 32), (unsigned)((pP + 31) / 32)), 256, 0, ctx->stream>>>(
        n, (int)p, M, ld, e, nK, KT, pP, S);
    count_launch(ctx, 3);
  };
  slice(X, ldx, pa, paP, ex, SX);
  if (!same) slice(Y, ldy, pb, pyP, ey, SY);

  OzArgs a{};
  a.SA = SX;
  a.SB = SY;
  a.rowsA = paP;
  a.rowsB = pyP;
  a.mode = 0;
  a.chunks = KT / OZ_KC;
  a.half_chunks = nK / OZ_KC;
  a.n_im0 = C == 2 ? pbP : (1 << 30);
  a.tiles = dtiles;
  a.H = H;
  a.L = L;
  a.NP = NP;
  const int ntiles = (int)tiles.size();
  int64_t nsplit = pick_splits(ntiles, a.chunks, ctx->num_sms);
  a.chunks_per_split = (a.chunks + nsplit - 1) / nsplit;
  nsplit = (a.chunks + a.chunks_per_split - 1) / a.chunks_per_split;
  launch_oz(ctx, a, ntiles, (int)nsplit);
  k_oz_gram_finish<T><<<(unsigned)((pa * pb + 255) / 256), 256, 0, ctx->stream>>>(
      (int)pa, (int)pb, pbP, NP, C == 2 ? pbP : 0, hermitian, H, L, ex, ey, G, ldg);
  count_launch(ctx);
}
template void gram_tc<double>(apf_ctx*, int64_t, int64_t, int64_t, const double*, int64_t, const double*, int64_t,
                              double*, int64_t, bool);
template void gram_tc<double2>(apf_ctx*, int64_t, int64_t, int64_t, const double2*, int64_t, const double2*,
                               int64_t, double2*, int64_t, bool);

template <class T>
void gemm_tall_tc(apf_ctx* ctx, int64_t n, int64_t pa, int64_t pb, const T* X, int64_t ldx, const T* M, int64_t ldm,
                  T* Z, int64_t ldz, double alpha, double beta, const T* Z0, int64_t ldz0) {
  if (n == 0 || pb == 0) return;
  constexpr int C = ScalarTraits<T>::is_complex ? 2 : 1;
  APF_REQUIRE(pa >= 1 && pa <= APF_MAX_P && pb <= APF_MAX_P, APF_ERR_ARG);
  const int64_t KT = round_up(C * pa, OZ_KC);
  const int64_t nP = round_up(n, OZ_BM);
  const int NT = (int)round_up(C * pb, OZ_NQ);
  const size_t sa = (size_t)OZS * nP * KT * 2, sb = (size_t)OZS * NT * KT * 2;
  const int ntm = (int)(nP / OZ_BM);
  std::vector<OzTile> tiles;
  for (int tm = 0; tm < ntm; ++tm) push_tiles(tiles, tm * OZ_BM, 0, NT);
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off = round_up((int64_t)(off + b), 1024); return o; };
  const size_t o_sa = take(sa), o_sb = take(sb), o_ea = take((size_t)nP * 4), o_fb = take((size_t)NT * 4);
  const size_t o_t = take(tiles.size() * sizeof(OzTile));
  unsigned char* ws = static_cast<unsigned char*>(workspace(ctx, off));
  auto* SA = reinterpret_cast<__nv_bfloat16*>(ws + o_sa);
  auto* SB = reinterpret_cast<__nv_bfloat16*>(ws + o_sb);
  int* ea = reinterpret_cast<int*>(ws + o_ea);
  int* fb = reinterpret_cast<int*>(ws + o_fb);
  OzTile* dtiles = reinterpret_cast<OzTile*>(ws + o_t);
  APF_CUDA(cudaMemcpyAsync(dtiles, tiles.data(), tiles.size() * sizeof(OzTile), cudaMemcpyHostToDevice,
                           ctx->stream));
  k_ozt_rowexp<T, C><<<(unsigned)((nP + 7) / 8), 256, 0, ctx->stream>>>(n, (int)pa, X, ldx, nP, ea);
  k_ozt_split_rows<T, C><<<(unsigned)((nP * KT + 255) / 256), 256, 0, ctx->stream>>>(n, (int)pa, X, ldx, ea, nP, KT,
                                                                                     SA);
  k_ozt_split_small<T, C><<<(unsigned)NT, 256, 0, ctx->stream>>>((int)pa, (int)pb, M, ldm, NT, KT, SB, fb);
  count_launch(ctx, 3);
  OzArgs a{};
  a.SA = SA;
  a.SB = SB;
  a.rowsA = nP;
  a.rowsB = NT;
  a.mode = 1;
  a.chunks = KT / OZ_KC;
  a.chunks_per_split = a.chunks;
  a.tiles = dtiles;
  a.n_im0 = 1 << 30;
  a.nrows = n;
  a.ncols = C * (int)pb;
  a.pb = (int)pb;
  a.cplx = C == 2;
  a.ea = ea;
  a.fb = fb;
  a.Z = reinterpret_cast<double*>(Z);
  a.Z0 = reinterpret_cast<const double*>(Z0 ? Z0 : Z);
  a.ldz = ldz;
  a.ldz0 = Z0 ? ldz0 : ldz;
  a.alpha = alpha;
  a.beta = Z0 ? beta : 0.0;
  APF_REQUIRE(tiles.size() <= (size_t)INT32_MAX, APF_ERR_ARG);
  launch_oz(ctx, a, (int)tiles.size(), 1);
}
template void gemm_tall_tc<double>(apf_ctx*, int64_t, int64_t, int64_t, const double*, int64_t, const double*,
                                   int64_t, double*, int64_t, double, double, const double*, int64_t);
template void gemm_tall_tc<double2>(apf_ctx*, int64_t, int64_t, int64_t, const double2*, int64_t, const double2*,
                                    int64_t, double2*, int64_t, double, double, const double2*, int64_t);

}  // namespace apf
