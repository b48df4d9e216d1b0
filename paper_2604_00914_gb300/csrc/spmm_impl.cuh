// The fused Clenshaw step: one sparse-times-dense-block product with the
// recurrence's axpy terms in the epilogue (Alg. 2, loop body):
//
//     Out[i,:] = alpha * sum_j A[i,j] W[j,:]  -  Vin[i,:]  +  f .* Y[i,:]
//
// Layout: A in CSR (int64 row pointers, int32 columns, values of type TA);
// W, Vin, Y, Out are row-major n x ld blocks.  A group of G threads owns one
// row; each thread owns VPT 16-byte column vectors of that row, so a row of
// the block is read and written with contiguous 16-byte accesses.  The group
// loads G nonzeros at a time (one per lane) and broadcasts them with warp
// shuffles; every nonzero then gathers one row of W (neighbouring rows of a
// banded matrix hit in L2).  Y and Vin stream through once (evict-first),
// accumulation is in T's precision.
#pragma once
#include "apf_internal.h"

namespace apf {

template <class T>
union Pack16 {
  uint4 u;
  T t[ScalarTraits<T>::per16];
};

template <class TA>
__device__ __forceinline__ TA shfl_g(TA v, int src, int G, unsigned mask);
template <>
__device__ __forceinline__ double shfl_g<double>(double v, int src, int G, unsigned mask) {
  return __shfl_sync(mask, v, src, G);
}
template <>
__device__ __forceinline__ float shfl_g<float>(float v, int src, int G, unsigned mask) {
  return __shfl_sync(mask, v, src, G);
}
template <>
__device__ __forceinline__ double2 shfl_g<double2>(double2 v, int src, int G, unsigned mask) {
  return make_double2(__shfl_sync(mask, v.x, src, G), __shfl_sync(mask, v.y, src, G));
}
template <>
__device__ __forceinline__ float2 shfl_g<float2>(float2 v, int src, int G, unsigned mask) {
  return make_float2(__shfl_sync(mask, v.x, src, G), __shfl_sync(mask, v.y, src, G));
}

template <class T, class TA, int G, int VPT>
__global__ void __launch_bounds__(256)
k_clenshaw_step(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                const TA* __restrict__ vals, const T* __restrict__ W, const T* Vin,
                const T* __restrict__ Y, int64_t ld, int nvec,
                const typename ScalarTraits<T>::Real* __restrict__ coef_col,
                typename ScalarTraits<T>::Real coef_scalar, typename ScalarTraits<T>::Real alpha,
                T* Out) {
  using Real = typename ScalarTraits<T>::Real;
  constexpr int E = ScalarTraits<T>::per16;
  const int lane = threadIdx.x % G;
  const int group_in_warp = (threadIdx.x % 32) / G;
  const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (group_in_warp * G));
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G;
  const bool valid = row < n;

  T acc[VPT][E];
#pragma unroll
  for (int q = 0; q < VPT; ++q)
#pragma unroll
    for (int e = 0; e < E; ++e) acc[q][e] = szero<T>();

  const int64_t s = valid ? rowptr[row] : 0;
  const int64_t eend = valid ? rowptr[row + 1] : 0;
  for (int64_t base = s; base < eend; base += G) {
    const int64_t idx = base + lane;
    int c_l = 0;
    TA v_l = szero<TA>();
    if (idx < eend) {
      c_l = __ldg(colidx + idx);
      v_l = __ldg(vals + idx);
    }
    const int cnt = (int)((eend - base) < G ? (eend - base) : G);
#pragma unroll 4
    for (int t = 0; t < cnt; ++t) {
      const int col = __shfl_sync(mask, c_l, t, G);
      const TA v = shfl_g<TA>(v_l, t, G, mask);
      const uint4* wrow = reinterpret_cast<const uint4*>(W + (int64_t)col * ld);
#pragma unroll
      for (int q = 0; q < VPT; ++q) {
        const int vi = lane + q * G;
        if (vi < nvec) {
          Pack16<T> w;
          w.u = __ldg(wrow + vi);
#pragma unroll
          for (int e = 0; e < E; ++e) madd(acc[q][e], v, w.t[e]);
        }
      }
    }
  }
  if (!valid) return;
  const int64_t rbase = row * ld;
#pragma unroll
  for (int q = 0; q < VPT; ++q) {
    const int vi = lane + q * G;
    if (vi >= nvec) continue;
    Pack16<T> y, v, o;
    y.u = make_uint4(0u, 0u, 0u, 0u);
    v.u = y.u;
    if (Y) y.u = __ldcs(reinterpret_cast<const uint4*>(Y + rbase) + vi);
    if (Vin) v.u = __ldcs(reinterpret_cast<const uint4*>(Vin + rbase) + vi);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const Real f = Y ? (coef_col ? coef_col[vi * E + e] : coef_scalar) : (Real)0;
      o.t[e] = step_out(acc[q][e], alpha, Vin != nullptr, v.t[e], Y != nullptr, f, y.t[e]);
    }
    reinterpret_cast<uint4*>(Out + rbase)[vi] = o.u;
  }
}

// (G, VPT) with the least idle lanes for nvec 16-byte vectors per row; ties go
// to more vectors per thread (fewer shuffles per useful load).
inline void choose_group(int nvec, int* G, int* VPT) {
  static const int gs[4] = {4, 8, 16, 32};
  static const int vs[7] = {1, 2, 3, 4, 5, 6, 8};
  int bestG = 32, bestV = 8;
  double best = 1e30;
  for (int gi = 0; gi < 4; ++gi)
    for (int vj = 0; vj < 7; ++vj) {
      const int g = gs[gi], v = vs[vj];
      if (g * v < nvec) continue;
      const double waste = (double)(g * v - nvec) / (g * v);
      const double score = waste * 100.0 - v * 0.01;
      if (score < best) { best = score; bestG = g; bestV = v; }
    }
  if (nvec > 32 * 8) { bestG = 32; bestV = 8; }
  *G = bestG;
  *VPT = bestV;
}

#define APF_CLEN_CASE(GG, VV)                                                                  \
  if (G == GG && VPT == VV) {                                                                  \
    k_clenshaw_step<T, TA, GG, VV><<<grid, 256, 0, ctx->stream>>>(                             \
        n, rowptr, colidx, vals, W + c0, Vin ? Vin + c0 : nullptr, Y ? Y + c0 : nullptr, ld,   \
        nv, coef_col ? coef_col + c0 : nullptr, coef_scalar, alpha, Out + c0);                 \
    launched = true;                                                                           \
  }

template <class T, class TA>
void clenshaw_step_impl(apf_ctx* ctx, int Gsel, int Vsel, int64_t n, const int64_t* rowptr, const int32_t* colidx,
                        const TA* vals, const T* W, const T* Vin, const T* Y, int64_t ld,
                        int64_t ncols, const typename ScalarTraits<T>::Real* coef_col,
                        typename ScalarTraits<T>::Real coef_scalar,
                        typename ScalarTraits<T>::Real alpha, T* Out) {
  constexpr int E = ScalarTraits<T>::per16;
  APF_REQUIRE(ld % E == 0, APF_ERR_ARG);
  APF_REQUIRE(W != Out, APF_ERR_ARG);
  if (n == 0 || ncols == 0) return;
  const int64_t nvec_total = (ncols + E - 1) / E;
  APF_REQUIRE(nvec_total * E <= ld, APF_ERR_ARG);
  // very wide blocks are processed in column slabs of at most 256 vectors
  for (int64_t v0 = 0; v0 < nvec_total; v0 += 256) {
    const int nv = (int)((nvec_total - v0) < 256 ? (nvec_total - v0) : 256);
    const int64_t c0 = v0 * E;
    int G, VPT;
    choose_group(nv, &G, &VPT);
    if (Gsel > 0 && Vsel > 0 && Gsel * Vsel >= nv) { G = Gsel; VPT = Vsel; }
    const int64_t rows_per_block = 256 / G;
    const unsigned grid = (unsigned)((n + rows_per_block - 1) / rows_per_block);
    bool launched = false;
    APF_CLEN_CASE(4, 1) APF_CLEN_CASE(4, 2) APF_CLEN_CASE(4, 3) APF_CLEN_CASE(4, 4)
    APF_CLEN_CASE(4, 5) APF_CLEN_CASE(4, 6) APF_CLEN_CASE(4, 8)
    APF_CLEN_CASE(8, 1) APF_CLEN_CASE(8, 2) APF_CLEN_CASE(8, 3) APF_CLEN_CASE(8, 4)
    APF_CLEN_CASE(8, 5) APF_CLEN_CASE(8, 6) APF_CLEN_CASE(8, 8)
    APF_CLEN_CASE(16, 1) APF_CLEN_CASE(16, 2) APF_CLEN_CASE(16, 3) APF_CLEN_CASE(16, 4)
    APF_CLEN_CASE(16, 5) APF_CLEN_CASE(16, 6) APF_CLEN_CASE(16, 8)
    APF_CLEN_CASE(32, 1) APF_CLEN_CASE(32, 2) APF_CLEN_CASE(32, 3) APF_CLEN_CASE(32, 4)
    APF_CLEN_CASE(32, 5) APF_CLEN_CASE(32, 6) APF_CLEN_CASE(32, 8)
    APF_REQUIRE(launched, APF_ERR_ARG);
    count_launch(ctx);
  }
}

#undef APF_CLEN_CASE

}  // namespace apf
