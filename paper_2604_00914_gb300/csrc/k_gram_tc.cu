// G = X^H Y to FP64 accuracy on the tensor cores (the Gram products of the
// Cholesky QR and Rayleigh-Ritz steps of Alg. 4), by splitting FP64 into
// bf16 slices (the Ozaki scheme: Ozaki, Ogita, Oishi and Rump, Numer.
// Algorithms 59, 2012; with integer slices as in Ootomo, Ozaki and Yokota,
// IJHPCA 2024).
//
// Column a of X gets the exponent e_a with |x_ia| < 2^e_a (real and imaginary
// parts alike).  Each part is cut into S = 7 signed integer slices of at most
// 8 bits:  x_ia = 2^(e_a - 7) sum_s sigma_s 2^(-8 s) + r_ia, |r_ia| <= 2^(e_a - 56)
// (55 bits below 2^e_a: exact for entries within a factor 4 of the column's
// largest), sigma_s in [-128, 128], stored as bf16 (exact).  Then
//   sum_i x_ia y_ib = 2^(e_a + e_b - 14) sum_d 2^(-8 d) sum_{s + t = d} P_st,
// P_st = sum_i sigma_s(x_ia) sigma_t(y_ib), keeping d <= S - 1: with the
// remainders, the dropped terms are at most about 2^(e_a + e_b - 53) per row
// (worst case; random signs make the sum far smaller).  The P_st are sums
// of products of integers below 2^14: with d + 1 <= 7 slice pairs, the real
// and imaginary combinations (two products each) and 64 rows per chunk, every
// partial sum stays below 896 * 2^14 < 2^24, so the tensor cores' FP32
// accumulation is exact, in any order.  After each 64-row chunk the FP32 sums
// of each diagonal d are added, scaled by 2^(-8 d), into FP64 accumulators.
//
// Layout of the slices: [slice][part][column][row] with rows (the contracted
// index) contiguous, padded to a multiple of 64 rows and 32 columns with zeros,
// so that mma.sync.m16n8k16 (bf16, FP32 accumulate) reads A = X^H row-major
// and B = Y column-major straight from global memory.
#include <cuda_bf16.h>

#include "apf_internal.h"

namespace apf {

constexpr int OZ_S = 7;      // slices per part
constexpr int OZ_KC = 64;    // rows per exact FP32 chunk
constexpr int OZ_TILE = 32;  // output tile (OZ_TILE x OZ_TILE) per CTA of 4 warps

__device__ __forceinline__ double comp_abs_max(double v) { return fabs(v); }
__device__ __forceinline__ double comp_abs_max(double2 v) { return fmax(fabs(v.x), fabs(v.y)); }

template <class T>
__global__ void k_oz_colmax(int64_t n, int p, const T* __restrict__ X, int64_t ld, int64_t rows,
                            double* __restrict__ part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows, r1 = min(n, r0 + rows);
  double m = 0.0;
  for (int64_t i = r0; i < r1; ++i) m = fmax(m, comp_abs_max(X[i * ld + c]));
  part[(int64_t)blockIdx.y * p + c] = m;
}

__global__ void k_oz_exp(int p, int nb, const double* __restrict__ part, int* __restrict__ e) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p) return;
  double m = 0.0;
  for (int b = 0; b < nb; ++b) m = fmax(m, part[(int64_t)b * p + c]);
  int ex = 0;
  if (m > 0.0) frexp(m, &ex);  // m = f 2^ex, f in [0.5, 1): |x| <= m < 2^ex
  e[c] = ex;
}

// One 32 x 32 tile of X (rows i0.., columns a0..) through shared memory:
// read along the columns, write the slices along the rows.
template <class T, int C>
__global__ void __launch_bounds__(256)
k_oz_split(int64_t n, int p, const T* __restrict__ X, int64_t ld, const int* __restrict__ e, int64_t nK, int pP,
           __nv_bfloat16* __restrict__ S) {
  __shared__ __nv_bfloat16 tile[OZ_S][C][32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int a0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
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
    const int ex = (a < p) ? e[a] : 0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      double t = ldexp(part[c], -ex);  // |t| < 1
#pragma unroll
      for (int s = 0; s < OZ_S; ++s) {
        const double v = t * (s == 0 ? 128.0 : 256.0);
        const double sig = rint(v);    // |sig| <= 128
        t = v - sig;                   // exact, |t| <= 1/2
        tile[s][c][tx][r] = __float2bfloat16_rn((float)sig);
      }
    }
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {  // r: column within the tile now, tx: row
    const int a = a0 + r;
    const int64_t i = i0 + tx;
    if (a >= pP || i >= nK) continue;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s)
#pragma unroll
      for (int c = 0; c < C; ++c) S[(((int64_t)s * C + c) * pP + a) * nK + i] = tile[s][c][r][tx];
  }
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment (16 x 16, row-major, rows = output rows a, columns = k) at
// (a0, k0) of the slice matrix M (row stride nK elements)
__device__ __forceinline__ void load_a(const __nv_bfloat16* M, int64_t nK, int a0, int64_t k0, int lane,
                                       uint32_t* f) {
  const int g = lane >> 2, q = lane & 3;
  const uint32_t* r0 = reinterpret_cast<const uint32_t*>(M + (int64_t)(a0 + g) * nK + k0 + 2 * q);
  const uint32_t* r8 = reinterpret_cast<const uint32_t*>(M + (int64_t)(a0 + g + 8) * nK + k0 + 2 * q);
  f[0] = __ldg(r0);
  f[1] = __ldg(r8);
  f[2] = __ldg(r0 + 4);
  f[3] = __ldg(r8 + 4);
}
// B fragment (16 x 8, column-major: columns = output columns b, rows = k)
__device__ __forceinline__ void load_b(const __nv_bfloat16* M, int64_t nK, int b0, int64_t k0, int lane,
                                       uint32_t* f) {
  const int g = lane >> 2, q = lane & 3;
  const uint32_t* c0 = reinterpret_cast<const uint32_t*>(M + (int64_t)(b0 + g) * nK + k0 + 2 * q);
  f[0] = __ldg(c0);
  f[1] = __ldg(c0 + 4);
}

// Partial Gram of one 32 x 32 output tile over one row range: 4 warps, each
// 16 rows (a) x 16 columns (b, two n8 blocks).  part: FP64 [re, im] per entry
// (unscaled: the factor 2^(e_a + e_b - 14) is applied by the reduction).
template <int C>
__global__ void __launch_bounds__(128)
k_oz_gram(const __nv_bfloat16* __restrict__ XS, const __nv_bfloat16* __restrict__ YS, int64_t nK, int pPa, int pPb,
          int pa, int pb, int ntb, bool hermitian, int64_t rows_per_split, double* __restrict__ part) {
  int ta, tb;
  const int pid = blockIdx.x;
  if (hermitian) {
    int t = pid, a = 0;
    while (t >= ntb - a) { t -= ntb - a; ++a; }
    ta = a;
    tb = a + t;
  } else {
    ta = pid / ntb;
    tb = pid % ntb;
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int a0 = ta * OZ_TILE + (warp / 2) * 16;
  const int b0 = tb * OZ_TILE + (warp % 2) * 16;
  const int64_t k_begin = (int64_t)blockIdx.y * rows_per_split;
  const int64_t k_end = min(nK, k_begin + rows_per_split);
  const int64_t sliceX = (int64_t)C * pPa * nK, sliceY = (int64_t)C * pPb * nK;
  const int64_t partX = (int64_t)pPa * nK, partY = (int64_t)pPb * nK;

  double accR[2][4], accI[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int v = 0; v < 4; ++v) accR[j][v] = accI[j][v] = 0.0;

  for (int64_t kc = k_begin; kc < k_end; kc += OZ_KC) {
    double scale = 1.0;
#pragma unroll 1
    for (int d = 0; d < OZ_S; ++d) {
      float cR[2][4], cI[2][4];
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) cR[j][v] = cI[j][v] = 0.0f;
#pragma unroll 1
      for (int s = 0; s <= d; ++s) {
        const int t = d - s;
        const __nv_bfloat16* Ar = XS + s * sliceX;
        const __nv_bfloat16* Br = YS + t * sliceY;
#pragma unroll
        for (int kk = 0; kk < OZ_KC; kk += 16) {
          uint32_t ar[4], br[2][2];
          load_a(Ar, nK, a0, kc + kk, lane, ar);
          load_b(Br, nK, b0, kc + kk, lane, br[0]);
          load_b(Br, nK, b0 + 8, kc + kk, lane, br[1]);
          mma_bf16(cR[0], ar, br[0]);
          mma_bf16(cR[1], ar, br[1]);
          if constexpr (C == 2) {
            uint32_t ai[4], bi[2][2], nai[4];
            load_a(Ar + partX, nK, a0, kc + kk, lane, ai);
            load_b(Br + partY, nK, b0, kc + kk, lane, bi[0]);
            load_b(Br + partY, nK, b0 + 8, kc + kk, lane, bi[1]);
            // Re(conj(x) y) = xr yr + xi yi;  Im(conj(x) y) = xr yi - xi yr
            mma_bf16(cR[0], ai, bi[0]);
            mma_bf16(cR[1], ai, bi[1]);
            mma_bf16(cI[0], ar, bi[0]);
            mma_bf16(cI[1], ar, bi[1]);
#pragma unroll
            for (int v = 0; v < 4; ++v) nai[v] = ai[v] ^ 0x80008000u;  // -xi, exact
            mma_bf16(cI[0], nai, br[0]);
            mma_bf16(cI[1], nai, br[1]);
          }
        }
      }
      // exact integers below 2^24: scale by 2^(-8 d) and carry in FP64
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          accR[j][v] = fma((double)cR[j][v], scale, accR[j][v]);
          accI[j][v] = fma((double)cI[j][v], scale, accI[j][v]);
        }
      scale *= 1.0 / 256.0;
    }
  }
  const int g = lane >> 2, q = lane & 3;
  double* P = part + (int64_t)blockIdx.y * pa * pb * 2;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int ga = a0 + g + (v >= 2 ? 8 : 0);
      const int gb = b0 + j * 8 + 2 * q + (v & 1);
      if (ga < pa && gb < pb) {
        P[((int64_t)ga * pb + gb) * 2] = accR[j][v];
        P[((int64_t)ga * pb + gb) * 2 + 1] = accI[j][v];
      }
    }
}

template <class T>
__global__ void k_oz_reduce(int pa, int pb, int nsplit, bool hermitian, const double* __restrict__ part,
                            const int* __restrict__ ea, const int* __restrict__ eb, T* __restrict__ G,
                            int64_t ldg) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)pa * pb) return;
  const int i = (int)(idx / pb), j = (int)(idx % pb);
  const bool mirror = hermitian && (i / OZ_TILE > j / OZ_TILE);
  const int si = mirror ? j : i, sj = mirror ? i : j;
  double re = 0.0, im = 0.0;
  for (int k = 0; k < nsplit; ++k) {
    const double* P = part + (int64_t)k * pa * pb * 2 + ((int64_t)si * pb + sj) * 2;
    re += P[0];
    im += P[1];
  }
  const int sc = ea[si] + eb[sj] - 14;
  re = ldexp(re, sc);
  im = ldexp(im, sc);
  if (mirror) im = -im;
  if constexpr (ScalarTraits<T>::is_complex) G[(int64_t)i * ldg + j] = make_double2(re, im);
  else G[(int64_t)i * ldg + j] = re;
}

template <class T>
struct OzSlices {
  DBuf buf, ex;
  int64_t nK = 0;
  int pP = 0;
};

template <class T>
static void oz_split(apf_ctx* ctx, int64_t n, int64_t p, const T* X, int64_t ld, OzSlices<T>& o) {
  constexpr int C = ScalarTraits<T>::is_complex ? 2 : 1;
  o.nK = round_up(n, OZ_KC);
  o.pP = (int)round_up(p, OZ_TILE);
  o.buf.alloc((size_t)OZ_S * C * o.pP * o.nK * sizeof(__nv_bfloat16), ctx->stream, true);
  o.ex.alloc((size_t)o.pP * sizeof(int), ctx->stream, true);
  const int64_t nb = std::min<int64_t>(std::max<int64_t>(1, 4LL * ctx->num_sms), n);
  const int64_t rows = (n + nb - 1) / nb;
  DBuf part((size_t)nb * p * sizeof(double), ctx->stream, true);
  k_oz_colmax<T><<<dim3((unsigned)((p + 127) / 128), (unsigned)nb), 128, 0, ctx->stream>>>(n, (int)p, X, ld, rows,
                                                                                           part.as<double>());
  k_oz_exp<<<(unsigned)((p + 127) / 128), 128, 0, ctx->stream>>>((int)p, (int)nb, part.as<double>(), o.ex.template as<int>());
  k_oz_split<T, C><<<dim3((unsigned)(o.nK / 32), (unsigned)(o.pP / 32)), 256, 0, ctx->stream>>>(
      n, (int)p, X, ld, o.ex.template as<int>(), o.nK, o.pP, o.buf.template as<__nv_bfloat16>());
  count_launch(ctx, 3);
}

template <class T>
void gram_tc(apf_ctx* ctx, int64_t n, int64_t pa, int64_t pb, const T* X, int64_t ldx, const T* Y, int64_t ldy,
             T* G, int64_t ldg, bool hermitian) {
  if (pa == 0 || pb == 0) return;
  APF_REQUIRE(!hermitian || pa == pb, APF_ERR_ARG);
  APF_REQUIRE(n >= 1 && pa <= APF_MAX_P && pb <= APF_MAX_P, APF_ERR_ARG);
  constexpr int C = ScalarTraits<T>::is_complex ? 2 : 1;
  OzSlices<T> sx, sy;
  oz_split<T>(ctx, n, pa, X, ldx, sx);
  const bool same = (X == Y && ldx == ldy && pa == pb);
  if (!same) oz_split<T>(ctx, n, pb, Y, ldy, sy);
  const OzSlices<T>& oy = same ? sx : sy;
  const int nta = sx.pP / OZ_TILE, ntb = oy.pP / OZ_TILE;
  const int npairs = hermitian ? nta * (nta + 1) / 2 : nta * ntb;
  int64_t nsplit = (4LL * ctx->num_sms + npairs - 1) / npairs;
  const int64_t max_split = sx.nK / OZ_KC;
  nsplit = std::max<int64_t>(1, std::min(nsplit, max_split));
  int64_t rows = round_up((sx.nK + nsplit - 1) / nsplit, OZ_KC);
  nsplit = (sx.nK + rows - 1) / rows;
  DBuf part((size_t)nsplit * pa * pb * 2 * sizeof(double), ctx->stream, true);
  k_oz_gram<C><<<dim3((unsigned)npairs, (unsigned)nsplit), 128, 0, ctx->stream>>>(
      sx.buf.template as<__nv_bfloat16>(), oy.buf.template as<__nv_bfloat16>(), sx.nK, sx.pP, oy.pP, (int)pa, (int)pb, ntb, hermitian,
      rows, part.as<double>());
  k_oz_reduce<T><<<(unsigned)((pa * pb + 255) / 256), 256, 0, ctx->stream>>>(
      (int)pa, (int)pb, (int)nsplit, hermitian, part.as<double>(), sx.ex.template as<int>(), oy.ex.template as<int>(), G, ldg);
  count_launch(ctx, 2);
}
template void gram_tc<double>(apf_ctx*, int64_t, int64_t, int64_t, const double*, int64_t, const double*, int64_t,
                              double*, int64_t, bool);
template void gram_tc<double2>(apf_ctx*, int64_t, int64_t, int64_t, const double2*, int64_t, const double2*,
                               int64_t, double2*, int64_t, bool);

}  // namespace apf
