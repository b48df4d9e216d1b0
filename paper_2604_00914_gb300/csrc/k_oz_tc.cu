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
// rounding of F).  P_d over a chunk of 32 values of k is an integer below
// 7 x 32 x 2^14 < 2^22, so the tensor cores' FP32 accumulation is exact in
// any order.  After each chunk the seven FP32 sums are turned into integers
// exactly by adding 1.5 x 2^23 (the integer then sits in the low mantissa
// bits) and accumulated in 32-bit integers (at most 512 chunks per CTA keeps
// them below 2^31); at the end of the CTA they are folded into two 64-bit
// integers,  hi = P_0 2^16 + P_1 2^8 + P_2,  lo = P_3 2^24 + P_4 2^16 + P_5 2^8 + P_6,
// so C = 2^(E_m + F_n - 62) (hi 2^32 + lo) is formed once, in FP64.  (FP64
// arithmetic runs at a tiny fraction of the tensor rate on this part: the
// carry never touches it.)  Split-K partial sums are added with 64-bit
// integer atomics, which is exact and independent of the order.
//
// Kernel (one CTA per 128 x 32 output tile and K range, 320 threads):
//   warp 8  producer: per 32-wide k chunk, bulk copies (cp.async.bulk) of the
//           seven 128 x 32 digit tiles of A and the seven 32 x 32 tiles of B,
//           stored pre-swizzled (64-byte swizzle) in global memory, into a
//           three-stage ring;
//   warp 9  MMA issuer: 28 slice pairs x 2 k steps of tcgen05.mma
//           (M = 128, N = 32, K = 16, bf16 in, FP32 accumulate) into one of
//           two sets of seven TMEM accumulators (7 x 32 columns each);
//   warps 0-7  drain: read the accumulators with tcgen05.ld (warp w owns TMEM
//           lanes 32 (w mod 4) .. +31, i.e. rows of the tile, and columns
//           16 (w / 4) .. +15) and accumulate the integers.
// The stages and accumulator sets are handed over with mbarriers; every wait
// is bounded in time and a timeout makes all roles stop, let their copies
// land, free the TMEM and record DEV_BARRIER_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>

#include "apf_internal.h"
#include "spmm_sell.cuh"

namespace apf {

constexpr int OZS = 7;        // digits per value
constexpr int OZ_BM = 128;    // output tile rows (MMA M)
constexpr int OZ_BN = 32;     // output tile columns (MMA N)
constexpr int OZ_KC = 32;     // k per chunk (one 64-byte swizzle row of bf16)
constexpr int OZ_ACC = OZS * OZ_BN;        // TMEM columns of one accumulator set
constexpr uint32_t OZ_A_SLICE = OZ_BM * OZ_KC * 2;   // 8 KB
constexpr uint32_t OZ_B_SLICE = OZ_BN * OZ_KC * 2;   // 2 KB
constexpr uint32_t OZ_A_STAGE = OZS * OZ_A_SLICE;    // 56 KB
constexpr uint32_t OZ_B_STAGE = OZS * OZ_B_SLICE;    // 14 KB
constexpr int OZ_STAGES = 3;                        // operand ring depth
constexpr size_t OZ_SMEM = 1024 + OZ_STAGES * (size_t)(OZ_A_STAGE + OZ_B_STAGE) + 1024;

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

struct OzArgs {
  const __nv_bfloat16* SA;  // digit planes of A (rowsA rows) and B (rowsB rows)
  const __nv_bfloat16* SB;
  int64_t rowsA, rowsB;
  int mode;          // 0: Gram (int64 atomics into H, L); 1: tall product (FP64 out)
  int64_t chunks;    // k chunks of this product (KT / OZ_KC)
  int64_t chunks_per_split;
  int ntile_n;       // output tiles along n
  const int2* tiles; // (tile m, tile n) per blockIdx.x
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
constexpr int OZ_MAX_CHUNKS = 512;  // per CTA: keeps the 32-bit sums below 2^31

__global__ void __launch_bounds__(OZ_THREADS, 1)
k_oz_umma(OzArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1 KB-aligned operand area (the swizzle atoms need 512-byte alignment)
  const uint32_t base_s = smem_addr(smem_raw);
  unsigned char* smem = smem_raw + ((1024 - (base_s & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);        // [3] bulk copies -> MMA
  uint64_t* empty = full + OZ_STAGES;                         // [3] MMA -> producer
  uint64_t* tfull = empty + OZ_STAGES;                        // [2] MMA -> drain
  uint64_t* tempty = tfull + 2;                               // [2] drain -> MMA
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tempty + 3);
  unsigned char* opA = smem + 1024;
  unsigned char* opB = opA + OZ_STAGES * OZ_A_STAGE;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int2 tile = a.tiles[blockIdx.x];
  const int m0 = tile.x * OZ_BM, n0 = tile.y * OZ_BN;
  const int64_t c_begin = (int64_t)blockIdx.y * a.chunks_per_split;
  const int64_t c_end = min(a.chunks, c_begin + a.chunks_per_split);
  const int nch = (int)(c_end > c_begin ? c_end - c_begin : 0);

  if (threadIdx.x == 0) {
    for (int i = 0; i < OZ_STAGES; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull + i, 1);
      mbar_init(tempty + i, OZ_DRAIN);
    }
    *abort_flag = 0;
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

  if (warp == 8) {
    if (lane == 0) {
      const int nb = im_tile ? n0 - a.n_im0 : n0;
      for (int c = 0; c < nch; ++c) {
        const int st = c % OZ_STAGES, use = c / OZ_STAGES;
        if (c >= OZ_STAGES && !oz_wait(empty + st, (uint32_t)((use - 1) & 1), a.limit_ns, abort_flag)) break;
        const int64_t kc = c_begin + c;
        int64_t kb = kc;
        if (im_tile) kb = kc < a.half_chunks ? kc + a.half_chunks : kc - a.half_chunks;
        mbar_arrive_expect(full + st, OZ_A_STAGE + OZ_B_STAGE);
        for (int sl = 0; sl < OZS; ++sl) {
          bulk_g2s(opA + st * OZ_A_STAGE + sl * OZ_A_SLICE, a.SA + oz_off(kc, sl, m0, a.rowsA, 0), OZ_A_SLICE, full + st);
          bulk_g2s(opB + st * OZ_B_STAGE + sl * OZ_B_SLICE, a.SB + oz_off(kb, sl, nb, a.rowsB, 0), OZ_B_SLICE, full + st);
        }
      }
    }
  } else if (warp == 9) {
    if (lane == 0) {
      const uint32_t id_pos = umma_idesc(OZ_BM, OZ_BN, false);
      const uint32_t id_neg = umma_idesc(OZ_BM, OZ_BN, true);
      for (int c = 0; c < nch; ++c) {
        const int st = c % OZ_STAGES, b = c & 1;
        if (!oz_wait(full + st, (uint32_t)((c / OZ_STAGES) & 1), a.limit_ns, abort_flag)) break;
        if (c >= 2 && !oz_wait(tempty + b, (uint32_t)(((c >> 1) - 1) & 1), a.limit_ns, abort_flag)) break;
        tc_fence_after();
        const uint32_t idesc = (im_tile && c_begin + c >= a.half_chunks) ? id_neg : id_pos;
        // descriptors of the stage's first tiles; the other tiles are at fixed
        // offsets (the 14-bit address field holds addr / 16 and never carries)
        const uint64_t ad0 = umma_desc_sw64(smem_addr(opA + st * OZ_A_STAGE));
        const uint64_t bd0 = umma_desc_sw64(smem_addr(opB + st * OZ_B_STAGE));
        const uint32_t dt0 = tbase + (uint32_t)(b * OZ_ACC);
#pragma unroll
        for (int d = 0; d < OZS; ++d) {
#pragma unroll
          for (int s = 0; s <= d; ++s) {
#pragma unroll
            for (int kk = 0; kk < OZ_KC / 16; ++kk) {
              const uint64_t ad = ad0 + (uint64_t)((s * OZ_A_SLICE + kk * 32) >> 4);
              const uint64_t bd = bd0 + (uint64_t)(((d - s) * OZ_B_SLICE + kk * 32) >> 4);
              if (s == 0 && kk == 0) umma_bf16_first(dt0 + d * OZ_BN, ad, bd, idesc);
              else umma_bf16_acc(dt0 + d * OZ_BN, ad, bd, idesc);
            }
          }
        }
        umma_commit(empty + st);
        umma_commit(tfull + b);
      }
    }
  } else {
    // drain: thread = row 32 (warp mod 4) + lane of the tile, columns 16 (warp / 4) + 0..15
    constexpr int HC = OZ_BN / 2;
    const int quarter = warp & 3, half = warp >> 2;
    int acc[OZS][HC];
#pragma unroll
    for (int d = 0; d < OZS; ++d)
#pragma unroll
      for (int j = 0; j < HC; ++j) acc[d][j] = 0;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    // an exact FP32 integer v, |v| < 2^22: the bits of v + 1.5 2^23 are MAGIC + v
    constexpr float kMagicF = 12582912.0f;
    constexpr int kMagicI = 0x4B400000;
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
      const int b = c & 1;
      if (!oz_wait(tfull + b, (uint32_t)((c >> 1) & 1), a.limit_ns, abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      // two diagonals (16 columns each) per wait: the 112 sums stay in registers
#pragma unroll
      for (int d0 = 0; d0 < OZS; d0 += 2) {
        uint32_t r0[HC], r1[HC];
        tmem_ld16(tbase + lane_off + (uint32_t)(b * OZ_ACC + d0 * OZ_BN + half * HC), r0);
        if (d0 + 1 < OZS) tmem_ld16(tbase + lane_off + (uint32_t)(b * OZ_ACC + (d0 + 1) * OZ_BN + half * HC), r1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < HC; ++j)
          acc[d0][j] += __float_as_int(__fadd_rn(__uint_as_float(r0[j]), kMagicF)) - kMagicI;
        if (d0 + 1 < OZS)
#pragma unroll
          for (int j = 0; j < HC; ++j)
            acc[d0 + 1][j] += __float_as_int(__fadd_rn(__uint_as_float(r1[j]), kMagicF)) - kMagicI;
      }
      tc_fence_before();
      mbar_arrive(tempty + b);
    }
    if (ok && !*abort_flag) {
      // park the sums in the (now idle) operand area: the fold below then
      // needs few registers.  The last tfull wait means every MMA, hence every
      // read of the operand area and every TMA write into it, has completed.
      int* sacc = reinterpret_cast<int*>(opA) + threadIdx.x * (OZS * HC + 1);
#pragma unroll
      for (int d = 0; d < OZS; ++d)
#pragma unroll
        for (int j = 0; j < HC; ++j) sacc[d * HC + j] = acc[d][j];
      const int m = m0 + quarter * 32 + lane;
      const int nb0 = n0 + half * HC;
      auto fold = [&](int j, long long& hi, long long& lo) {
        hi = ((long long)sacc[0 * HC + j] << 16) + ((long long)sacc[1 * HC + j] << 8) + sacc[2 * HC + j];
        lo = ((long long)sacc[3 * HC + j] << 24) + ((long long)sacc[4 * HC + j] << 16) +
             ((long long)sacc[5 * HC + j] << 8) + sacc[6 * HC + j];
      };
      if (a.mode == 0) {
#pragma unroll 1
        for (int j = 0; j < HC; ++j) {
          long long hi, lo;
          fold(j, hi, lo);
          const int64_t o = (int64_t)m * a.NP + nb0 + j;
          if (hi) atomicAdd(a.H + o, (unsigned long long)hi);
          if (lo) atomicAdd(a.L + o, (unsigned long long)lo);
        }
      } else if (m < a.nrows) {
        const int em = a.ea[m];
#pragma unroll 1
        for (int j = 0; j < HC; ++j) {
          const int col = nb0 + j;
          if (col >= a.ncols) continue;
          long long hi, lo;
          fold(j, hi, lo);
          const int sc = em + a.fb[col] - 62;
          const double v = oz_scale((double)hi, sc + 32) + oz_scale((double)lo, sc);
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
    // the last stages' TMA copies and MMAs complete by themselves; wait for
    // their barriers (bounded) before the shared memory and TMEM go away
    if (threadIdx.x == 0) {
      volatile int dummy = 0;
      for (int c = (nch > OZ_STAGES ? nch - OZ_STAGES : 0); c < nch; ++c)
        oz_wait(full + c % OZ_STAGES, (uint32_t)((c / OZ_STAGES) & 1), 1000000000ull, &dummy);
      for (int c = (nch > 2 ? nch - 2 : 0); c < nch; ++c)
        oz_wait(tfull + (c & 1), (uint32_t)((c >> 1) & 1), 1000000000ull, &dummy);
    }
    __syncthreads();
  }
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

// hi/lo sums of the Gram -> G (FP64), mirroring the tiles below the diagonal
template <class T>
__global__ void k_oz_gram_finish(int pa, int pb, int NP, int n_im0, bool hermitian,
                                 const unsigned long long* __restrict__ H, const unsigned long long* __restrict__ L,
                                 const int* __restrict__ ea, const int* __restrict__ eb, T* __restrict__ G,
                                 int64_t ldg) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)pa * pb) return;
  const int i = (int)(idx / pb), j = (int)(idx % pb);
  // computed tiles: (tile m, tile n) with n range reaching the m range's start
  const bool have = !hermitian || (j / OZ_BN) * OZ_BN + OZ_BN - 1 >= (i / OZ_BM) * OZ_BM;
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
  APF_REQUIRE(a.chunks_per_split <= OZ_MAX_CHUNKS, APF_ERR_ARG);
  k_oz_umma<<<dim3((unsigned)ntiles, (unsigned)nsplit), OZ_THREADS, OZ_SMEM, ctx->stream>>>(a);
  count_launch(ctx);
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
  const int paP = (int)round_up(pa, OZ_BM), pbP = (int)round_up(pb, OZ_BN);
  const int NP = C * pbP;  // output columns: [re | im]
  const bool same = (X == Y && ldx == ldy && pa == pb);
  const int pyP = same ? paP : pbP;  // rows of Y's slice array
  // workspace: slices of X and Y, exponents, hi/lo sums, tile list, column maxima
  const int64_t nb = std::min<int64_t>(std::max<int64_t>(1, 4LL * ctx->num_sms), n);
  const int64_t rows_per = (n + nb - 1) / nb;
  const size_t sx = (size_t)OZS * paP * KT * 2, sy = same ? 0 : (size_t)OZS * pyP * KT * 2;
  const size_t hl = (size_t)paP * NP * 8;
  const int ntm = paP / OZ_BM, ntn = NP / OZ_BN;
  std::vector<int2> tiles;
  for (int tm = 0; tm < ntm; ++tm)
    for (int tn = 0; tn < ntn; ++tn) {
      const int b0 = (tn * OZ_BN) % pbP;
      if (hermitian && b0 + OZ_BN - 1 < tm * OZ_BM) continue;
      if (b0 >= pb) continue;  // padding columns only
      tiles.push_back(make_int2(tm, tn));
    }
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off = round_up((int64_t)(off + b), 1024); return o; };
  const size_t o_sx = take(sx), o_sy = take(sy), o_ex = take((size_t)paP * 4), o_ey = take((size_t)pyP * 4);
  const size_t o_h = take(hl), o_l = take(hl), o_t = take(tiles.size() * sizeof(int2));
  const size_t o_part = take((size_t)nb * std::max(pa, pb) * 8);
  unsigned char* ws = static_cast<unsigned char*>(workspace(ctx, off));
  auto* SX = reinterpret_cast<__nv_bfloat16*>(ws + o_sx);
  auto* SY = same ? SX : reinterpret_cast<__nv_bfloat16*>(ws + o_sy);
  int* ex = reinterpret_cast<int*>(ws + o_ex);
  int* ey = same ? ex : reinterpret_cast<int*>(ws + o_ey);
  auto* H = reinterpret_cast<unsigned long long*>(ws + o_h);
  auto* L = reinterpret_cast<unsigned long long*>(ws + o_l);
  int2* dtiles = reinterpret_cast<int2*>(ws + o_t);
  double* part = reinterpret_cast<double*>(ws + o_part);
  APF_CUDA(cudaMemcpyAsync(dtiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, ctx->stream));
  APF_CUDA(cudaMemsetAsync(H, 0, 2 * hl + (o_l - o_h - hl), ctx->stream));

  auto slice = [&](const T* M, int64_t ld, int64_t p, int pP, int* e, __nv_bfloat16* S) {
    k_ozt_colmax<T><<<dim3((unsigned)((p + 127) / 128), (unsigned)nb), 128, 0, ctx->stream>>>(n, (int)p, M, ld,
                                                                                           rows_per, part);
    k_ozt_colexp<<<(unsigned)((pP + 127) / 128), 128, 0, ctx->stream>>>((int)p, (int)nb, part, e, pP);
    k_ozt_split_cols<T, C><<<dim3((unsigned)(nK / 32), (unsigned)(pP / 32)), 256, 0, ctx->stream>>>(
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
  int64_t nsplit = (2LL * ctx->num_sms + ntiles - 1) / ntiles;
  nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, a.chunks / 8 > 0 ? a.chunks / 8 : 1));
  nsplit = std::max<int64_t>(nsplit, (a.chunks + OZ_MAX_CHUNKS - 1) / OZ_MAX_CHUNKS);
  a.chunks_per_split = (a.chunks + nsplit - 1) / nsplit;
  nsplit = (a.chunks + a.chunks_per_split - 1) / a.chunks_per_split;
  launch_oz(ctx, a, ntiles, (int)nsplit);
  k_oz_gram_finish<T><<<(unsigned)((pa * pb + 255) / 256), 256, 0, ctx->stream>>>(
      (int)pa, (int)pb, NP, C == 2 ? pbP : 0, hermitian, H, L, ex, ey, G, ldg);
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
  const int NT = (int)round_up(C * pb, OZ_BN);
  const size_t sa = (size_t)OZS * nP * KT * 2, sb = (size_t)OZS * NT * KT * 2;
  const int ntm = (int)(nP / OZ_BM), ntn = NT / OZ_BN;
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off = round_up((int64_t)(off + b), 1024); return o; };
  const size_t o_sa = take(sa), o_sb = take(sb), o_ea = take((size_t)nP * 4), o_fb = take((size_t)NT * 4);
  const size_t o_t = take((size_t)ntm * ntn * sizeof(int2));
  unsigned char* ws = static_cast<unsigned char*>(workspace(ctx, off));
  auto* SA = reinterpret_cast<__nv_bfloat16*>(ws + o_sa);
  auto* SB = reinterpret_cast<__nv_bfloat16*>(ws + o_sb);
  int* ea = reinterpret_cast<int*>(ws + o_ea);
  int* fb = reinterpret_cast<int*>(ws + o_fb);
  int2* dtiles = reinterpret_cast<int2*>(ws + o_t);
  std::vector<int2> tiles((size_t)ntm * ntn);
  for (int tm = 0; tm < ntm; ++tm)
    for (int tn = 0; tn < ntn; ++tn) tiles[(size_t)tm * ntn + tn] = make_int2(tm, tn);
  APF_CUDA(cudaMemcpyAsync(dtiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, ctx->stream));
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
  launch_oz(ctx, a, ntm * ntn, 1);
}
template void gemm_tall_tc<double>(apf_ctx*, int64_t, int64_t, int64_t, const double*, int64_t, const double*,
                                   int64_t, double*, int64_t, double, double, const double*, int64_t);
template void gemm_tall_tc<double2>(apf_ctx*, int64_t, int64_t, int64_t, const double2*, int64_t, const double2*,
                                    int64_t, double2*, int64_t, double, double, const double2*, int64_t);

}  // namespace apf
