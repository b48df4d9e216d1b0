// The Clenshaw step on the SELL-8 layout, one column tile per CTA.
//
// The one-CTA-per-row-range kernel (spmm_sell.cuh) gathers whole rows of W.
// For a matrix whose rows reach far (a 3D stencil on an L^3 grid touches rows
// +-4 L^2 away), the rows of W that a window of in-flight rows needs span
// 2 x 4 L^2 rows of the full block width; when that exceeds L2, every far
// neighbour is read from HBM again (measured: 11.8 GB of DRAM traffic against
// 4.5 GB of algorithmic bytes per step at 96^3 and width 300).
//
// Here the block's columns are cut into tiles of TV = G x VPT 16-byte vectors
// and the grid is (row ranges) x (column tiles), row ranges fastest, so the
// GPU sweeps the whole matrix once per column tile: the window of W that L2
// must hold shrinks by the number of tiles, and A's structure (a few per cent
// of the bytes) is read once per tile instead.  A tile also has no upper
// limit on the block width, which the batched spectrum slices need.  Which
// kernel is faster depends on the matrix and the width: in a cold single
// launch at 96^3 the tiles cut DRAM traffic to 6.2 GB and the time by 14 %,
// while in the back-to-back steps of a solve the one-tile kernel was faster
// there; the autotuner times both on the live buffers.
//
// Per CTA (R = 256 / G rows): one thread issues a 2-D TMA tensor copy of the
// R x TV tile of Y and of Vin (rows beyond n and columns beyond the block read
// as zero) and bulk copies of the rows' structure, completing on one mbarrier;
// the W rows are gathered into registers meanwhile.  Each row sums its entries
// in CSR order and the epilogue is the same fused operation as in the other
// kernels, so every variant gives the same bits.  Waits are bounded in time.
//
// Near rows (halo H > 0): the rows of a stencil's own grid line sit within a
// few rows of the diagonal, so the R rows of a CTA share them.  With a halo the
// CTA also copies rows r0 - H .. r0 + R + H - 1 of W's tile into shared memory
// (one more 2-D TMA copy; rows outside the matrix read as zero) and reads the
// entries whose column falls there from shared memory instead of L2: for the
// 25-point stencil of a 3D eighth-order Laplacian, 9 of the 25 gathered rows.
// The values read are the same, so the bits are too.
#pragma once
#include <cuda.h>

#include "spmm_sell.cuh"
#include "tma.h"

namespace apf {

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// shared-memory bytes of one CTA: barrier, Y and Vin tiles, near rows of W, structure
inline size_t sell_ct_smem_bytes(int R, int TV, int lmax, size_t sTA, int halo = 0) {
  size_t b = 128 + 2 * (size_t)R * TV * 16;
  if (halo > 0) b += (size_t)(R + 2 * halo) * TV * 16;
  b += (size_t)R * lmax * 4;
  b = (b + 15) / 16 * 16;
  b += (size_t)R * lmax * sTA;
  b += (size_t)(R / SELL_C + 1) * 8 + 16;
  return b;
}

template <class T, class TA, int G, int VPT>
__global__ void __launch_bounds__(256, (VPT <= 2 ? 4 : 3))
k_clenshaw_sell_ct(int64_t n, const int64_t* __restrict__ chunk_ptr, const int32_t* __restrict__ scol,
                   const TA* __restrict__ sval, int lmax, const T* __restrict__ W,
                   const __grid_constant__ CUtensorMap tmV, const __grid_constant__ CUtensorMap tmY,
                   const __grid_constant__ CUtensorMap tmW, int halo, int has_v,
                   int has_y, int64_t ld, int nvec, const typename ScalarTraits<T>::Real* __restrict__ coef_col,
                   typename ScalarTraits<T>::Real coef_scalar, typename ScalarTraits<T>::Real alpha,
                   T* __restrict__ Out, int* err, uint64_t limit_ns) {
  using Real = typename ScalarTraits<T>::Real;
  constexpr int E = ScalarTraits<T>::per16;
  constexpr int R = 256 / G;
  constexpr int TV = G * VPT;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  uint4* Ys = reinterpret_cast<uint4*>(smem + 128);
  uint4* Vs = Ys + R * TV;
  uint4* Ws = Vs + R * TV;                 // near rows of W (halo > 0)
  const int wn = halo > 0 ? R + 2 * halo : 0;
  int32_t* cols = reinterpret_cast<int32_t*>(Ws + wn * TV);
  size_t voff = (size_t)((unsigned char*)(cols + R * lmax) - smem);
  voff = (voff + 15) / 16 * 16;
  TA* vals = reinterpret_cast<TA*>(smem + voff);
  int64_t* cps = reinterpret_cast<int64_t*>(vals + R * lmax);

  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int v0 = blockIdx.y * TV;  // first vector of the tile
  const int nr = (int)((n - r0) < R ? (n - r0) : R);
  const int64_t c0 = r0 / SELL_C;
  const int nch = (nr + SELL_C - 1) / SELL_C;

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    const uint32_t tile = (uint32_t)(R * TV * 16);
    const uint32_t yv = (has_y ? tile : 0u) + (has_v ? tile : 0u) + (uint32_t)(wn * TV * 16);
    if (yv) mbar_expect_tx(bar, yv);
    // x in 4-byte units (the maps describe the block as floats)
    if (has_y) tma_load_2d(Ys, &tmY, v0 * 4, (int)r0, bar);
    if (has_v) tma_load_2d(Vs, &tmV, v0 * 4, (int)r0, bar);
    if (wn) tma_load_2d(Ws, &tmW, v0 * 4, (int)r0 - halo, bar);
    for (int c = 0; c <= nch; ++c) cps[c] = chunk_ptr[c0 + c];
    const int64_t e0 = cps[0], e1 = cps[nch];
    const uint32_t nc = (uint32_t)((e1 - e0) * 4), nv = (uint32_t)((e1 - e0) * sizeof(TA));
    mbar_expect_tx(bar, nc + nv);
    bulk_g2s(cols, scol + e0, nc, bar);
    bulk_g2s(vals, sval + e0, nv, bar);
    mbar_arrive(bar);
  }
  __syncthreads();  // barrier initialised, cps written
  const bool landed = mbar_wait_bounded(bar, 0u, limit_ns);
  if (!__syncthreads_and(landed)) {
    if (threadIdx.x == 0) atomicCAS(err, 0, DEV_BARRIER_TIMEOUT);
    mbar_wait_bounded(bar, 0u, limit_ns > 1000000000ull ? limit_ns : 1000000000ull);
    return;
  }

  const int lane = threadIdx.x % G;
  const int rl = threadIdx.x / G;
  if (rl >= nr) return;
  const int64_t row = r0 + rl;
  const int cl = rl / SELL_C, rr = rl % SELL_C;
  const int64_t base = cps[cl] - cps[0];
  const int len = (int)((cps[cl + 1] - cps[cl]) / SELL_C);

  T acc[VPT][E];
#pragma unroll
  for (int q = 0; q < VPT; ++q)
#pragma unroll
    for (int e = 0; e < E; ++e) acc[q][e] = szero<T>();

  const int wlo = (int)r0 - halo;
#pragma unroll 4
  for (int t = 0; t < len; ++t) {
    const int64_t s = base + (int64_t)t * SELL_C + rr;
    const int col = cols[s];
    const TA v = vals[s];
    const unsigned rel = (unsigned)(col - wlo);
    const bool near = rel < (unsigned)wn;
    const uint4* wrow = near ? Ws + (int64_t)rel * TV : reinterpret_cast<const uint4*>(W + (int64_t)col * ld) + v0;
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
      const int vl = lane + q * G;
      if (v0 + vl < nvec) {
        Pack16<T> w;
        w.u = near ? wrow[vl] : __ldg(wrow + vl);
#pragma unroll
        for (int e = 0; e < E; ++e) madd(acc[q][e], v, w.t[e]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < VPT; ++q) {
    const int vl = lane + q * G;
    const int vi = v0 + vl;
    if (vi >= nvec) continue;
    Pack16<T> y, v, o;
    y.u = Ys[rl * TV + vl];
    v.u = Vs[rl * TV + vl];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const Real f = has_y ? (coef_col ? coef_col[vi * E + e] : coef_scalar) : (Real)0;
      o.t[e] = step_out(acc[q][e], alpha, has_v != 0, v.t[e], has_y != 0, f, y.t[e]);
    }
    reinterpret_cast<uint4*>(Out + row * ld)[vi] = o.u;
  }
}

// The (G, VPT) shapes compiled for the column-tiled kernel: tiles of 8, 16,
// 32 and 64 vectors (128 B to 1 KB of a row).
static const SellShape kSellCtShapes[] = {{8, 1}, {8, 2}, {16, 1}, {8, 4}, {16, 2}, {32, 1},
                                          {16, 4}, {32, 2}};

template <class T, class TA>
void clenshaw_sell_ct_launch(apf_ctx* ctx, int G, int VPT, int64_t n, const int64_t* chunk_ptr,
                             const int32_t* scol, const TA* sval, int lmax, const T* W, const T* Vin,
                             const T* Y, int64_t ld, int64_t ncols,
                             const typename ScalarTraits<T>::Real* coef_col,
                             typename ScalarTraits<T>::Real coef_scalar,
                             typename ScalarTraits<T>::Real alpha, T* Out, int halo = 0) {
  constexpr int E = ScalarTraits<T>::per16;
  APF_REQUIRE(ld % E == 0 && W != Out, APF_ERR_ARG);
  if (n == 0 || ncols == 0) return;
  const int nvec = (int)((ncols + E - 1) / E);
  const int R = 256 / G, TV = G * VPT;
  APF_REQUIRE(n <= INT32_MAX && (int64_t)nvec * E <= ld, APF_ERR_ARG);
  APF_REQUIRE(halo >= 0 && R + 2 * halo <= 256, APF_ERR_ARG);
  const size_t smem = sell_ct_smem_bytes(R, TV, lmax, sizeof(TA), halo);
  APF_REQUIRE(smem <= 200 * 1024, APF_ERR_ARG);
  // the blocks as n x (ld * sizeof(T) / 4) floats, boxes of TV vectors x R rows
  const uint64_t inner = (uint64_t)ld * sizeof(T) / 4;
  CUtensorMap mv, my, mw;
  memset(&mv, 0, sizeof(mv));
  memset(&my, 0, sizeof(my));
  memset(&mw, 0, sizeof(mw));
  if (halo > 0)
    APF_REQUIRE(encode_tmap_2d(&mw, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, W, inner, (uint64_t)n, ld * sizeof(T),
                               (uint32_t)(TV * 4), (uint32_t)(R + 2 * halo), CU_TENSOR_MAP_SWIZZLE_NONE),
                APF_ERR_CUDA);
  if (Vin)
    APF_REQUIRE(encode_tmap_2d(&mv, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, Vin, inner, (uint64_t)n, ld * sizeof(T),
                               (uint32_t)(TV * 4), (uint32_t)R, CU_TENSOR_MAP_SWIZZLE_NONE),
                APF_ERR_CUDA);
  if (Y)
    APF_REQUIRE(encode_tmap_2d(&my, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, Y, inner, (uint64_t)n, ld * sizeof(T),
                               (uint32_t)(TV * 4), (uint32_t)R, CU_TENSOR_MAP_SWIZZLE_NONE),
                APF_ERR_CUDA);
  const dim3 grid((unsigned)((n + R - 1) / R), (unsigned)((nvec + TV - 1) / TV));
  APF_REQUIRE(grid.y <= 65535, APF_ERR_ARG);
  const int hv = Vin != nullptr, hy = Y != nullptr;
  bool launched = false;
#define APF_SELL_CT_CASE(GG, VV)                                                                    \
  if (G == GG && VPT == VV) {                                                                       \
    allow_large_smem<k_clenshaw_sell_ct<T, TA, GG, VV>>(ctx->device);                              \
    k_clenshaw_sell_ct<T, TA, GG, VV><<<grid, 256, smem, ctx->stream>>>(                            \
        n, chunk_ptr, scol, sval, lmax, W, mv, my, mw, halo, hv, hy, ld, nvec, coef_col, coef_scalar,  \
        alpha, Out, ctx->d_err, filter_wait_ns(ctx));                                               \
    launched = true;                                                                                \
  }
  APF_SELL_CT_CASE(8, 1) APF_SELL_CT_CASE(8, 2) APF_SELL_CT_CASE(16, 1) APF_SELL_CT_CASE(8, 4)
  APF_SELL_CT_CASE(16, 2) APF_SELL_CT_CASE(32, 1) APF_SELL_CT_CASE(16, 4) APF_SELL_CT_CASE(32, 2)
#undef APF_SELL_CT_CASE
  APF_REQUIRE(launched, APF_ERR_ARG);
  count_launch(ctx);
}

}  // namespace apf
