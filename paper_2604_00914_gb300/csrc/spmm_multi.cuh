// One Clenshaw step (Alg. 2) for several independent problems in one launch:
// the serving engine's batched filter step.
//
// Each problem r (its own matrix A_r in SELL-8 form, its own blocks) is given
// by a descriptor: structure, the step's W, Vin, Y and Out buffers, leading
// dimension, width, coefficients (per column or one scalar) and alpha.  The
// grid is the concatenation of every problem's tiles, problem by problem; a
// tile is R = 256 / G consecutive rows and one column tile of TV = G x VPT
// 16-byte vectors, row ranges fastest within a problem.  A CTA finds its
// problem by a scan over at most kMaxBatch tile offsets, stages its rows'
// structure with two bulk copies (mbarrier, bounded wait), gathers W into
// registers and reads Y and Vin straight from global memory in the epilogue.
// The arithmetic (entries summed in CSR order, the fused round-to-nearest
// epilogue) is that of every other step kernel, so a problem's result does
// not depend on which other problems share the launch.
#pragma once
#include "spmm_sell.cuh"

namespace apf {

constexpr int kMaxBatch = 16;

struct MultiDesc {
  const int64_t* chunk_ptr;
  const int32_t* scol;
  const void* sval;
  const void* W;
  const void* Vin;   // nullptr: no V term
  const void* Y;     // nullptr: no Y term
  void* Out;
  const float* coef_col;  // nullptr: coef_scalar for every column
  float coef_scalar, alpha;
  int64_t n, ld;
  int nvec, lmax, tile0, nrt, nct;
};

struct MultiArgs {
  int nreq, total_tiles;
  MultiDesc d[kMaxBatch];
  int* err;
  uint64_t limit_ns;
};

inline size_t multi_smem_bytes(int R, int lmax, size_t sTA) {
  size_t b = 128 + (size_t)R * lmax * 4;
  b = (b + 15) / 16 * 16;
  b += (size_t)R * lmax * sTA;
  b += (size_t)(R / SELL_C + 1) * 8 + 16;
  return b;
}

template <class T, class TA, int G, int VPT>
__global__ void __launch_bounds__(256, 4) k_clenshaw_multi(const __grid_constant__ MultiArgs a) {
  using Real = typename ScalarTraits<T>::Real;
  constexpr int E = ScalarTraits<T>::per16;
  constexpr int R = 256 / G;
  constexpr int TV = G * VPT;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);

  int r = 0;
  for (int q = 1; q < a.nreq; ++q)
    if ((int)blockIdx.x >= a.d[q].tile0) r = q;
  const MultiDesc& d = a.d[r];
  const int t = (int)blockIdx.x - d.tile0;
  const int ct = t / d.nrt, rt = t % d.nrt;
  const int64_t r0 = (int64_t)rt * R;
  const int v0 = ct * TV;
  const int64_t n = d.n;
  const int lmax = d.lmax;
  int32_t* cols = reinterpret_cast<int32_t*>(smem + 128);
  size_t voff = (size_t)((unsigned char*)(cols + R * lmax) - smem);
  voff = (voff + 15) / 16 * 16;
  TA* vals = reinterpret_cast<TA*>(smem + voff);
  int64_t* cps = reinterpret_cast<int64_t*>(vals + R * lmax);

  const int nr = (int)((n - r0) < R ? (n - r0) : R);
  const int64_t c0 = r0 / SELL_C;
  const int nch = (nr + SELL_C - 1) / SELL_C;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    for (int c = 0; c <= nch; ++c) cps[c] = d.chunk_ptr[c0 + c];
    const int64_t e0 = cps[0], e1 = cps[nch];
    const uint32_t nc = (uint32_t)((e1 - e0) * 4), nv = (uint32_t)((e1 - e0) * sizeof(TA));
    mbar_expect_tx(bar, nc + nv);
    bulk_g2s(cols, d.scol + e0, nc, bar);
    bulk_g2s(vals, static_cast<const TA*>(d.sval) + e0, nv, bar);
    mbar_arrive(bar);
  }
  __syncthreads();
  const bool landed = mbar_wait_bounded(bar, 0u, a.limit_ns);
  if (!__syncthreads_and(landed)) {
    if (threadIdx.x == 0) atomicCAS(a.err, 0, DEV_BARRIER_TIMEOUT);
    mbar_wait_bounded(bar, 0u, a.limit_ns > 1000000000ull ? a.limit_ns : 1000000000ull);
    return;
  }

  const int lane = threadIdx.x % G;
  const int rl = threadIdx.x / G;
  if (rl >= nr) return;
  const int64_t row = r0 + rl;
  const int cl = rl / SELL_C, rr = rl % SELL_C;
  const int64_t base = cps[cl] - cps[0];
  const int len = (int)((cps[cl + 1] - cps[cl]) / SELL_C);
  const T* W = static_cast<const T*>(d.W);
  const int64_t ld = d.ld;
  const int nvec = d.nvec;

  T acc[VPT][E];
#pragma unroll
  for (int q = 0; q < VPT; ++q)
#pragma unroll
    for (int e = 0; e < E; ++e) acc[q][e] = szero<T>();

#pragma unroll 4
  for (int tt = 0; tt < len; ++tt) {
    const int64_t s = base + (int64_t)tt * SELL_C + rr;
    const int col = cols[s];
    const TA v = vals[s];
    const uint4* wrow = reinterpret_cast<const uint4*>(W + (int64_t)col * ld) + v0;
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
      const int vl = lane + q * G;
      if (v0 + vl < nvec) {
        Pack16<T> w;
        w.u = __ldg(wrow + vl);
#pragma unroll
        for (int e = 0; e < E; ++e) madd(acc[q][e], v, w.t[e]);
      }
    }
  }
  const bool hv = d.Vin != nullptr, hy = d.Y != nullptr;
  const uint4* yrow = hy ? reinterpret_cast<const uint4*>(static_cast<const T*>(d.Y) + row * ld) : nullptr;
  const uint4* vrow = hv ? reinterpret_cast<const uint4*>(static_cast<const T*>(d.Vin) + row * ld) : nullptr;
  uint4* orow = reinterpret_cast<uint4*>(static_cast<T*>(d.Out) + row * ld);
#pragma unroll
  for (int q = 0; q < VPT; ++q) {
    const int vi = v0 + lane + q * G;
    if (vi >= nvec) continue;
    Pack16<T> y, v, o;
    y.u = make_uint4(0u, 0u, 0u, 0u);
    v.u = y.u;
    if (hy) y.u = __ldcs(yrow + vi);
    if (hv) v.u = __ldcs(vrow + vi);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const Real f = hy ? (d.coef_col ? (Real)d.coef_col[vi * E + e] : (Real)d.coef_scalar) : (Real)0;
      o.t[e] = step_out(acc[q][e], (Real)d.alpha, hv, v.t[e], hy, f, y.t[e]);
    }
    orow[vi] = o.u;
  }
}

// the batched step's tile shape: 32 rows x 16 vectors (64 floats or 32 complex)
constexpr int kMultiG = 8, kMultiVPT = 2;

// Launch one batched step for the problems in a (tile0 / nrt / nct filled here).
template <class T>
void clenshaw_multi_launch(apf_ctx* ctx, MultiArgs& a) {
  constexpr int R = 256 / kMultiG, TV = kMultiG * kMultiVPT;
  constexpr int E = ScalarTraits<T>::per16;
  APF_REQUIRE(a.nreq >= 1 && a.nreq <= kMaxBatch, APF_ERR_ARG);
  int tiles = 0, lmax = 1;
  for (int r = 0; r < a.nreq; ++r) {
    MultiDesc& d = a.d[r];
    APF_REQUIRE(d.ld % E == 0 && (int64_t)d.nvec * E <= d.ld && d.W != d.Out, APF_ERR_ARG);
    d.tile0 = tiles;
    d.nrt = (int)((d.n + R - 1) / R);
    d.nct = (d.nvec + TV - 1) / TV;
    APF_REQUIRE((int64_t)tiles + (int64_t)d.nrt * d.nct < INT32_MAX, APF_ERR_ARG);
    tiles += d.nrt * d.nct;
    lmax = d.lmax > lmax ? d.lmax : lmax;
  }
  if (tiles == 0) return;
  a.total_tiles = tiles;
  a.err = ctx->d_err;
  a.limit_ns = filter_wait_ns(ctx);
  const size_t smem = multi_smem_bytes(R, lmax, sizeof(T));
  APF_REQUIRE(smem <= 200 * 1024, APF_ERR_ARG);
  allow_large_smem<k_clenshaw_multi<T, T, kMultiG, kMultiVPT>>(ctx->device);
  k_clenshaw_multi<T, T, kMultiG, kMultiVPT><<<(unsigned)tiles, 256, smem, ctx->stream>>>(a);
  count_launch(ctx);
}

}  // namespace apf
