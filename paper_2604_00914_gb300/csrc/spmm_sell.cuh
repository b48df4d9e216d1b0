// The Clenshaw step on the SELL-8 layout with TMA bulk-copy staging.
//
// Layout (built at ingest, SELL-C-sigma with C = 8, sigma = 1: rows keep their
// order): chunk c holds rows 8c..8c+7, padded to the chunk's longest row;
// entry t of row r sits at chunk_ptr[c] + 8 t + (r mod 8).  Padding entries
// point at the row itself with value 0, so they add exact zeros.
//
// A CTA owns R = 256 / G consecutive rows, i.e. R / 8 whole chunks whose
// entries are one contiguous range.  At kernel start one thread issues
// cp.async.bulk copies (TMA, completion on an mbarrier) of that range's
// column indices and values and of the CTA's rows of Y and Vin (contiguous,
// row-major) into shared memory; the rows of W are then gathered into
// registers (neighbouring rows of a banded matrix hit in L2) while the copies
// are in flight, and the epilogue reads Y and Vin from shared memory.  The
// dependent chain per row is thus: one round for the structure (overlapped
// with the Y / Vin staging), the gathers, the store.
//
// Every wait on the mbarrier is bounded in time (limit_ns, a kernel argument:
// 1 s unless the context sets another); on expiry the kernel records
// DEV_BARRIER_TIMEOUT, waits (bounded) for its copies and returns.
#pragma once
#include <atomic>

#include "spmm_impl.cuh"

namespace apf {

constexpr int SELL_C = 8;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ uint64_t sell_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for a phase of the CTA's barrier.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = sell_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (sell_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// shared-memory bytes of one CTA: barrier, staged Y and Vin rows, structure
inline size_t sell_smem_bytes(int R, int64_t ld, size_t sT, int lmax, size_t sTA, bool y, bool vin) {
  size_t b = 128;
  b += (y ? (size_t)R * ld * sT : 0) + (vin ? (size_t)R * ld * sT : 0);
  b += (size_t)R * lmax * 4;
  b = (b + 15) / 16 * 16;
  b += (size_t)R * lmax * sTA;
  b += (size_t)(R / SELL_C + 1) * 8 + 16;
  return b;
}

struct NoWait {
  __device__ bool operator()() const { return true; }
};

// One tile of R = 256 / G rows starting at r0: stage structure, Y and Vin with
// bulk copies on `bar` (phase `parity`), call wait() (all threads; it may
// block until other tiles are done), gather W, write Out.  W is read through
// the non-coherent path unless COHERENT_W (data written earlier in the same
// launch).  Returns false after a timeout (recorded in err).
template <class T, class TA, int G, int VPT, bool COHERENT_W, class Wait>
__device__ __forceinline__ bool sell_tile(
    int64_t r0, int64_t n, const int64_t* __restrict__ chunk_ptr, const int32_t* __restrict__ scol,
    const TA* __restrict__ sval, int lmax, const T* W, const T* Vin, const T* Y, int64_t ld, int nvec,
    const typename ScalarTraits<T>::Real* __restrict__ coef_col, typename ScalarTraits<T>::Real coef_scalar,
    typename ScalarTraits<T>::Real alpha, T* Out, unsigned char* smem, uint64_t* bar, uint32_t parity,
    int* err, uint64_t limit_ns, const Wait& wait) {
  using Real = typename ScalarTraits<T>::Real;
  constexpr int E = ScalarTraits<T>::per16;
  constexpr int R = 256 / G;
  T* Ys = reinterpret_cast<T*>(smem + 128);
  T* Vs = Ys + (Y ? (int64_t)R * ld : 0);
  int32_t* cols = reinterpret_cast<int32_t*>(Vs + (Vin ? (int64_t)R * ld : 0));
  size_t voff = (size_t)((unsigned char*)(cols + R * lmax) - smem);
  voff = (voff + 15) / 16 * 16;
  TA* vals = reinterpret_cast<TA*>(smem + voff);
  int64_t* cps = reinterpret_cast<int64_t*>(vals + R * lmax);

  const int nr = (int)((n - r0) < R ? (n - r0) : R);
  const int64_t c0 = r0 / SELL_C;
  const int nch = (nr + SELL_C - 1) / SELL_C;

  if (threadIdx.x == 0) {
    uint32_t yv = 0;
    if (Y) yv += (uint32_t)((int64_t)nr * ld * sizeof(T));
    if (Vin) yv += (uint32_t)((int64_t)nr * ld * sizeof(T));
    if (yv) mbar_expect_tx(bar, yv);
    if (Y) bulk_g2s(Ys, Y + r0 * ld, (uint32_t)((int64_t)nr * ld * sizeof(T)), bar);
    if (Vin) bulk_g2s(Vs, Vin + r0 * ld, (uint32_t)((int64_t)nr * ld * sizeof(T)), bar);
    for (int c = 0; c <= nch; ++c) cps[c] = chunk_ptr[c0 + c];
    const int64_t e0 = cps[0], e1 = cps[nch];
    const uint32_t nc = (uint32_t)((e1 - e0) * 4), nv = (uint32_t)((e1 - e0) * sizeof(TA));
    mbar_expect_tx(bar, nc + nv);
    bulk_g2s(cols, scol + e0, nc, bar);
    bulk_g2s(vals, sval + e0, nv, bar);
    mbar_arrive(bar);
  }
  const bool ready = wait();
  const bool landed = mbar_wait_bounded(bar, parity, limit_ns);
  if (!__syncthreads_and(ready && landed)) {  // one decision for the whole CTA
    if (threadIdx.x == 0) atomicCAS(err, 0, DEV_BARRIER_TIMEOUT);
    // let the copies land before leaving (they complete by themselves; the
    // limit is at least the default so a short test limit cannot cut it off)
    mbar_wait_bounded(bar, parity, limit_ns > 1000000000ull ? limit_ns : 1000000000ull);
    return false;
  }

  const int lane = threadIdx.x % G;
  const int rl = threadIdx.x / G;  // local row
  if (rl >= nr) return true;
  const int64_t row = r0 + rl;
  const int cl = rl / SELL_C, rr = rl % SELL_C;
  const int64_t base = cps[cl] - cps[0];
  const int len = (int)((cps[cl + 1] - cps[cl]) / SELL_C);

  T acc[VPT][E];
#pragma unroll
  for (int q = 0; q < VPT; ++q)
#pragma unroll
    for (int e = 0; e < E; ++e) acc[q][e] = szero<T>();

#pragma unroll 4
  for (int t = 0; t < len; ++t) {
    const int64_t s = base + (int64_t)t * SELL_C + rr;
    const int col = cols[s];
    const TA v = vals[s];
    const uint4* wrow = reinterpret_cast<const uint4*>(W + (int64_t)col * ld);
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
      const int vi = lane + q * G;
      if (vi < nvec) {
        Pack16<T> w;
        // written earlier in this launch by other CTAs: load from L2, never
        // from this SM's L1, which may hold a line fetched before the rows
        // next to the waited-for range were written
        if constexpr (COHERENT_W) w.u = __ldcg(wrow + vi);
        else w.u = __ldg(wrow + vi);
#pragma unroll
        for (int e = 0; e < E; ++e) madd(acc[q][e], v, w.t[e]);
      }
    }
  }
  const T* ys = Ys + (int64_t)rl * ld;
  const T* vs = Vs + (int64_t)rl * ld;
#pragma unroll
  for (int q = 0; q < VPT; ++q) {
    const int vi = lane + q * G;
    if (vi >= nvec) continue;
    Pack16<T> y, v, o;
    y.u = make_uint4(0u, 0u, 0u, 0u);
    v.u = y.u;
    if (Y) y.u = reinterpret_cast<const uint4*>(ys)[vi];
    if (Vin) v.u = reinterpret_cast<const uint4*>(vs)[vi];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const Real f = Y ? (coef_col ? coef_col[vi * E + e] : coef_scalar) : (Real)0;
      o.t[e] = step_out(acc[q][e], alpha, Vin != nullptr, v.t[e], Y != nullptr, f, y.t[e]);
    }
    reinterpret_cast<uint4*>(Out + row * ld)[vi] = o.u;
  }
  return true;
}

// Four CTAs per SM up to VPT = 6 (64 registers, no spills): more warps in
// flight to cover the gathers of W; measured 4.7 % faster than three at
// 64^3, p = 160.
template <class T, class TA, int G, int VPT>
__global__ void __launch_bounds__(256, (VPT <= 6 ? 4 : 2))
k_clenshaw_sell(int64_t n, const int64_t* __restrict__ chunk_ptr, const int32_t* __restrict__ scol,
                const TA* __restrict__ sval, int lmax, const T* __restrict__ W, const T* Vin,
                const T* __restrict__ Y, int64_t ld, int nvec,
                const typename ScalarTraits<T>::Real* __restrict__ coef_col,
                typename ScalarTraits<T>::Real coef_scalar, typename ScalarTraits<T>::Real alpha, T* Out,
                int* err, uint64_t limit_ns) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  constexpr int R = 256 / G;
  sell_tile<T, TA, G, VPT, false>((int64_t)blockIdx.x * R, n, chunk_ptr, scol, sval, lmax, W, Vin, Y, ld,
                                  nvec, coef_col, coef_scalar, alpha, Out, smem, bar, 0u, err, limit_ns,
                                  NoWait());
}

// ---- two Clenshaw steps in one pass (temporal blocking) -----------------------------
//
//   step 1 (tile t):  B[t] = 2 A_hat A_ - Va + f1 .* Y      (b_j from b_{j+1} = A, b_{j+2} = Va)
//   step 2 (tile t):  A[t] = 2 A_hat B  - A  + f2 .* Y      (b_{j-1} from b_j = B, b_{j+1} = A)
//
// A persistent grid walks the work items in a fixed order in which step 2 of
// tile t comes after step 1 of every tile that it reads (t +- halo tiles) and
// that reads what it overwrites: step 1 of tile u reads rows of A within the
// bandwidth of tile u, so once step 1 is done on all tiles within t +- halo,
// A[t] may be overwritten.  Items are dealt round-robin to the CTAs, each CTA
// takes its items in order, and a step-2 item waits (bounded in time) until the
// step-1 counters of the 32-tile segments it depends on reach this pass; every
// item it waits for sits earlier in the order, so the waits always end.  The
// rows of B and Y that step 2 reads were touched by step 1 a few hundred tiles
// earlier and still sit in L2: the pass moves A_, Va and Y in and B and A out
// (5 block streams) where two single steps move 8.
constexpr int PAIR_SEG = 32;

struct PairDeps {
  const unsigned* seg_count;
  int t, halo, ntiles;
  unsigned pass;
  uint64_t limit_ns;
  __device__ bool operator()() const {
    const int lo = (t - halo > 0 ? t - halo : 0) / PAIR_SEG;
    const int hi = (t + halo < ntiles - 1 ? t + halo : ntiles - 1) / PAIR_SEG;
    const uint64_t t0 = sell_ns();
    for (;;) {
      bool mine = true;
      for (int s = lo + (int)threadIdx.x; s <= hi; s += (int)blockDim.x) {
        const int first = s * PAIR_SEG;
        const int cnt = (ntiles - first) < PAIR_SEG ? (ntiles - first) : PAIR_SEG;
        const unsigned have = *(volatile const unsigned*)(seg_count + s);
        if (have < pass * (unsigned)cnt) mine = false;
      }
      if (__syncthreads_and(mine)) break;
      if (__syncthreads_or(sell_ns() - t0 > limit_ns)) return false;
      __nanosleep(128);
    }
    __threadfence();
    return true;
  }
};

struct PairArgs {
  int64_t n;
  const int64_t* chunk_ptr;
  const int32_t* scol;
  const void* sval;
  int lmax;
  void* bufA;        // b_{j+1} in, b_{j-1} out
  void* bufB;        // b_j out (may equal va)
  const void* va;    // b_{j+2} (nullptr: zero)
  const void* Y;
  int64_t ld;
  int nvec;
  const void* coef1_col;
  double coef1;
  const void* coef2_col;
  double coef2;
  int ntiles, halo, lag;
  unsigned* seg_count;
  unsigned pass;
  int* err;
  uint64_t limit_ns;
};

__device__ __forceinline__ void pair_item(int q, int ntiles, int lag, int* kind, int* t) {
  const int D = lag < ntiles ? lag : ntiles;
  if (q < D) { *kind = 1; *t = q; return; }
  const int q2 = q - D, m = ntiles - D;
  if (q2 < 2 * m) {
    if ((q2 & 1) == 0) { *kind = 1; *t = D + q2 / 2; }
    else { *kind = 2; *t = q2 / 2; }
    return;
  }
  *kind = 2;
  *t = m + (q2 - 2 * m);
}

template <class T, class TA, int G, int VPT>
__global__ void __launch_bounds__(256, (VPT <= 6 ? 4 : 2))
k_clenshaw_sell_pair(PairArgs a) {
  using Real = typename ScalarTraits<T>::Real;
  constexpr int R = 256 / G;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  T* A = static_cast<T*>(a.bufA);
  T* Bb = static_cast<T*>(a.bufB);
  const T* Va = static_cast<const T*>(a.va);
  const T* Y = static_cast<const T*>(a.Y);
  const TA* sval = static_cast<const TA*>(a.sval);
  const Real* f1 = static_cast<const Real*>(a.coef1_col);
  const Real* f2 = static_cast<const Real*>(a.coef2_col);
  uint32_t parity = 0;
  const int total = 2 * a.ntiles;
  for (int q = blockIdx.x; q < total; q += gridDim.x) {
    int kind, t;
    pair_item(q, a.ntiles, a.lag, &kind, &t);
    const int64_t r0 = (int64_t)t * R;
    bool ok;
    if (kind == 1) {
      ok = sell_tile<T, TA, G, VPT, false>(r0, a.n, a.chunk_ptr, a.scol, sval, a.lmax, A, Va, Y, a.ld, a.nvec,
                                           f1, (Real)a.coef1, (Real)2, Bb, smem, bar, parity, a.err, a.limit_ns,
                                           NoWait());
    } else {
      PairDeps deps{a.seg_count, t, a.halo, a.ntiles, a.pass, a.limit_ns};
      ok = sell_tile<T, TA, G, VPT, true>(r0, a.n, a.chunk_ptr, a.scol, sval, a.lmax, Bb, A, Y, a.ld, a.nvec,
                                          f2, (Real)a.coef2, (Real)2, A, smem, bar, parity, a.err, a.limit_ns,
                                          deps);
    }
    parity ^= 1u;
    if (!ok) return;
    __syncthreads();
    if (kind == 1 && threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.seg_count + t / PAIR_SEG, 1u);
    }
  }
}

// The (G, VPT) shapes compiled for the SELL kernel.
struct SellShape {
  int G, VPT;
};
static const SellShape kSellShapes[] = {{8, 1}, {8, 2}, {8, 3}, {8, 4}, {16, 2}, {16, 3}, {16, 4},
                                        {16, 5}, {16, 6}, {32, 2}, {32, 3}, {32, 4}, {32, 5}, {32, 6},
                                        {32, 8}};

// Opt a kernel into 200 KB of dynamic shared memory, once per device; safe to
// call from several host threads (contexts may live on different threads).
template <auto Kern>
inline void allow_large_smem(int device) {
  static std::atomic<uint64_t> done{0};
  const uint64_t bit = 1ull << (device & 63);
  if (done.load(std::memory_order_acquire) & bit) return;
  APF_CUDA(cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  done.fetch_or(bit, std::memory_order_release);
}

// The same for an explicit number of bytes.
template <auto Kern>
inline void allow_large_smem_bytes(int device, int bytes) {
  static std::atomic<uint64_t> done{0};
  const uint64_t bit = 1ull << (device & 63);
  if (done.load(std::memory_order_acquire) & bit) return;
  APF_CUDA(cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit, std::memory_order_release);
}

template <class T, class TA>
void clenshaw_sell_launch(apf_ctx* ctx, int G, int VPT, int64_t n, const int64_t* chunk_ptr,
                          const int32_t* scol, const TA* sval, int lmax, const T* W, const T* Vin,
                          const T* Y, int64_t ld, int64_t ncols,
                          const typename ScalarTraits<T>::Real* coef_col,
                          typename ScalarTraits<T>::Real coef_scalar,
                          typename ScalarTraits<T>::Real alpha, T* Out) {
  constexpr int E = ScalarTraits<T>::per16;
  APF_REQUIRE(ld % E == 0 && W != Out, APF_ERR_ARG);
  if (n == 0 || ncols == 0) return;
  const int nvec = (int)((ncols + E - 1) / E);
  APF_REQUIRE(nvec <= G * VPT, APF_ERR_ARG);
  const int R = 256 / G;
  const size_t smem = sell_smem_bytes(R, ld, sizeof(T), lmax, sizeof(TA), Y != nullptr, Vin != nullptr);
  APF_REQUIRE(smem <= 200 * 1024, APF_ERR_ARG);
  const unsigned grid = (unsigned)((n + R - 1) / R);
  bool launched = false;
#define APF_SELL_CASE(GG, VV)                                                                        \
  if (G == GG && VPT == VV) {                                                                        \
    auto kern = k_clenshaw_sell<T, TA, GG, VV>;                                                      \
    allow_large_smem<k_clenshaw_sell<T, TA, GG, VV>>(ctx->device);                                   \
    kern<<<grid, 256, smem, ctx->stream>>>(n, chunk_ptr, scol, sval, lmax, W, Vin, Y, ld, nvec,      \
                                           coef_col, coef_scalar, alpha, Out, ctx->d_err,            \
                                           filter_wait_ns(ctx));                                     \
    launched = true;                                                                                 \
  }
  APF_SELL_CASE(8, 1) APF_SELL_CASE(8, 2) APF_SELL_CASE(8, 3) APF_SELL_CASE(8, 4)
  APF_SELL_CASE(16, 2) APF_SELL_CASE(16, 3) APF_SELL_CASE(16, 4) APF_SELL_CASE(16, 5) APF_SELL_CASE(16, 6)
  APF_SELL_CASE(32, 2) APF_SELL_CASE(32, 3) APF_SELL_CASE(32, 4) APF_SELL_CASE(32, 5) APF_SELL_CASE(32, 6)
  APF_SELL_CASE(32, 8)
#undef APF_SELL_CASE
  APF_REQUIRE(launched, APF_ERR_ARG);
  count_launch(ctx);
}

// Two steps in one cooperative launch (every CTA resident, which the ordered
// waits rely on).  seg_count: ceil(ntiles / 32) counters, zero before the first
// pass of a buffer set; `pass` counts the passes made with them (from 1).
template <class T, class TA>
void clenshaw_sell_pair_launch(apf_ctx* ctx, int G, int VPT, int64_t n, const int64_t* chunk_ptr,
                               const int32_t* scol, const TA* sval, int lmax, int64_t bandwidth, T* bufA,
                               T* bufB, const T* va, const T* Y, int64_t ld, int64_t ncols,
                               const typename ScalarTraits<T>::Real* coef1_col,
                               typename ScalarTraits<T>::Real coef1,
                               const typename ScalarTraits<T>::Real* coef2_col,
                               typename ScalarTraits<T>::Real coef2, unsigned* seg_count, unsigned pass) {
  constexpr int E = ScalarTraits<T>::per16;
  APF_REQUIRE(ld % E == 0 && bufA != bufB && Y != nullptr, APF_ERR_ARG);
  if (n == 0 || ncols == 0) return;
  const int nvec = (int)((ncols + E - 1) / E);
  APF_REQUIRE(nvec <= G * VPT, APF_ERR_ARG);
  const int R = 256 / G;
  const size_t smem = sell_smem_bytes(R, ld, sizeof(T), lmax, sizeof(TA), true, true);
  APF_REQUIRE(smem <= 200 * 1024, APF_ERR_ARG);
  PairArgs a;
  a.n = n;
  a.chunk_ptr = chunk_ptr;
  a.scol = scol;
  a.sval = sval;
  a.lmax = lmax;
  a.bufA = bufA;
  a.bufB = bufB;
  a.va = va;
  a.Y = Y;
  a.ld = ld;
  a.nvec = nvec;
  a.coef1_col = coef1_col;
  a.coef1 = (double)coef1;
  a.coef2_col = coef2_col;
  a.coef2 = (double)coef2;
  a.ntiles = (int)((n + R - 1) / R);
  a.halo = (int)((bandwidth + R - 1) / R);
  a.seg_count = seg_count;
  a.pass = pass;
  a.err = ctx->d_err;
  a.limit_ns = filter_wait_ns(ctx);
  bool launched = false;
#define APF_PAIR_CASE(GG, VV)                                                                         \
  if (G == GG && VPT == VV) {                                                                         \
    auto kern = k_clenshaw_sell_pair<T, TA, GG, VV>;                                                  \
    allow_large_smem<k_clenshaw_sell_pair<T, TA, GG, VV>>(ctx->device);                               \
    int per_sm = 0;                                                                                   \
    APF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));                \
    APF_REQUIRE(per_sm >= 1, APF_ERR_ARG);                                                            \
    int grid = per_sm * ctx->num_sms;                                                                 \
    if (grid > 2 * a.ntiles) grid = 2 * a.ntiles;                                                     \
    /* step 2 of a tile trails step 1 by the halo, a segment, and the items in flight */             \
    a.lag = a.halo + PAIR_SEG + 1 + grid;                                                             \
    void* args[] = {&a};                                                                              \
    APF_CUDA(cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(256), args, smem, ctx->stream)); \
    launched = true;                                                                                  \
  }
  APF_PAIR_CASE(8, 1) APF_PAIR_CASE(8, 2) APF_PAIR_CASE(8, 3) APF_PAIR_CASE(8, 4)
  APF_PAIR_CASE(16, 2) APF_PAIR_CASE(16, 3) APF_PAIR_CASE(16, 4) APF_PAIR_CASE(16, 5) APF_PAIR_CASE(16, 6)
  APF_PAIR_CASE(32, 2) APF_PAIR_CASE(32, 3) APF_PAIR_CASE(32, 4) APF_PAIR_CASE(32, 5) APF_PAIR_CASE(32, 6)
  APF_PAIR_CASE(32, 8)
#undef APF_PAIR_CASE
  APF_REQUIRE(launched, APF_ERR_ARG);
  count_launch(ctx);
}

}  // namespace apf
