// Small dense FP64 factorisations on p x p matrices (p <= APF_MAX_P):
//  - Cholesky G = R^H R (one CTA, right-looking), for Cholesky QR (Alg. 4);
//  - inverse of an upper triangular R (one warp per column);
//  - Hermitian eigendecomposition for Rayleigh-Ritz (Alg. 1) and for the
//    Lanczos tridiagonal matrix: one-sided (Hestenes) Jacobi on M = B + sI,
//    s = 2 ||B||_inf, so that M is positive definite with condition <= 3.
//    For a positive definite M the orthogonalised columns of M V are
//    sigma_j u_j with u_j the eigenvectors, so only M is rotated.  Column
//    pairs follow the round-robin (circle) ordering: each round has P/2
//    disjoint pairs, one warp per pair, and the rounds are separated by a
//    grid barrier of a cooperative launch.  The barrier gives up after a
//    fixed wall time and reports DEV_BARRIER_TIMEOUT instead of spinning on.
#include <cooperative_groups.h>

#include "apf_internal.h"

namespace apf {

__device__ __forceinline__ void set_err(int* err, int code) { atomicCAS(err, 0, code); }
__device__ __forceinline__ double rabs(double v) { return fabs(v); }
__device__ __forceinline__ double rabs(double2 v) { return hypot(v.x, v.y); }

// ---- Cholesky ---------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(1024) k_cholesky_upper(int p, T* G, int64_t ldg, double shift,
                                                         int* err) {
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid / 32, lane = tid % 32, nwarps = nt / 32;
  if (tid == 0) fail = 0;
  if (shift != 0.0)
    for (int i = tid; i < p; i += nt) G[(int64_t)i * ldg + i] = add(G[(int64_t)i * ldg + i], make_val<T>(shift, 0.0));
  __syncthreads();
  for (int k = 0; k < p; ++k) {
    if (tid == 0) {
      const double d = real_(G[(int64_t)k * ldg + k]);
      if (!(d > 0.0) || !isfinite(d)) {
        fail = 1;
        set_err(err, DEV_CHOL_PIVOT);
      } else {
        G[(int64_t)k * ldg + k] = make_val<T>(sqrt(d), 0.0);
      }
    }
    __syncthreads();
    if (fail) return;
    const double r = real_(G[(int64_t)k * ldg + k]);
    const double rinv = 1.0 / r;
    for (int j = k + 1 + tid; j < p; j += nt) G[(int64_t)k * ldg + j] = rmul(rinv, G[(int64_t)k * ldg + j]);
    __syncthreads();
    for (int i = k + 1 + warp; i < p; i += nwarps) {
      const T gki = conj_(G[(int64_t)k * ldg + i]);
      for (int j = i + lane; j < p; j += 32) {
        T v = G[(int64_t)i * ldg + j];
        const T t = mul(gki, G[(int64_t)k * ldg + j]);
        G[(int64_t)i * ldg + j] = sub(v, t);
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < p * p; e += nt) {
    const int i = e / p, j = e % p;
    if (i > j) G[(int64_t)i * ldg + j] = szero<T>();
  }
}

template <class T>
void cholesky_upper(apf_ctx* ctx, int64_t p, T* G, int64_t ldg, double shift) {
  if (p == 0) return;
  k_cholesky_upper<T><<<1, 1024, 0, ctx->stream>>>((int)p, G, ldg, shift, ctx->d_err);
  count_launch(ctx);
}
template void cholesky_upper<double>(apf_ctx*, int64_t, double*, int64_t, double);
template void cholesky_upper<double2>(apf_ctx*, int64_t, double2*, int64_t, double);

// ---- inverse of an upper triangular matrix: column j solves R z = e_j --------
__device__ __forceinline__ double rdiv(double a, double b) { return a / b; }
__device__ __forceinline__ double2 rdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

template <class T>
__global__ void k_tri_inv_upper(int p, const T* __restrict__ R, int64_t ldr, T* __restrict__ Ri,
                                int64_t ldri) {
  extern __shared__ unsigned char smem_raw[];
  T* z = reinterpret_cast<T*>(smem_raw);
  const int j = blockIdx.x, lane = threadIdx.x;
  for (int i = lane; i < p; i += 32) z[i] = szero<T>();
  __syncwarp();
  if (lane == 0) z[j] = rdiv(make_val<T>(1.0, 0.0), R[(int64_t)j * ldr + j]);
  __syncwarp();
  for (int i = j - 1; i >= 0; --i) {
    T s = szero<T>();
    for (int k = i + 1 + lane; k <= j; k += 32) madd(s, R[(int64_t)i * ldr + k], z[k]);
    s = warp_sum(s);
    if (lane == 0) z[i] = rdiv(sub(szero<T>(), s), R[(int64_t)i * ldr + i]);
    __syncwarp();
  }
  for (int i = lane; i < p; i += 32) Ri[(int64_t)i * ldri + j] = z[i];
}

template <class T>
void tri_inv_upper(apf_ctx* ctx, int64_t p, const T* R, int64_t ldr, T* Rinv, int64_t ldri) {
  if (p == 0) return;
  k_tri_inv_upper<T><<<(unsigned)p, 32, (size_t)p * sizeof(T), ctx->stream>>>((int)p, R, ldr, Rinv, ldri);
  count_launch(ctx);
}
template void tri_inv_upper<double>(apf_ctx*, int64_t, const double*, int64_t, double*, int64_t);
template void tri_inv_upper<double2>(apf_ctx*, int64_t, const double2*, int64_t, double2*, int64_t);

// ---- B <- (B + B^H)/2 -------------------------------------------------------------
template <class T>
__global__ void k_symmetrize(int p, T* B, int64_t ldb) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)p * p) return;
  const int i = (int)(e / p), j = (int)(e % p);
  if (i > j) return;
  const T a = B[(int64_t)i * ldb + j], b = conj_(B[(int64_t)j * ldb + i]);
  T m = rmul(0.5, add(a, b));
  if (i == j) m = make_val<T>(real_(m), 0.0);
  B[(int64_t)i * ldb + j] = m;
  B[(int64_t)j * ldb + i] = conj_(m);
}

template <class T>
void symmetrize(apf_ctx* ctx, int64_t p, T* B, int64_t ldb) {
  if (p == 0) return;
  k_symmetrize<T><<<(unsigned)((p * p + 255) / 256), 256, 0, ctx->stream>>>((int)p, B, ldb);
  count_launch(ctx);
}
template void symmetrize<double>(apf_ctx*, int64_t, double*, int64_t);
template void symmetrize<double2>(apf_ctx*, int64_t, double2*, int64_t);

// ---- ||B||_inf -------------------------------------------------------------------------
template <class T>
__global__ void k_inf_norm(int p, const T* __restrict__ B, int64_t ldb, double* out) {
  __shared__ double sm[256];
  double m = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < p; ++j) s += rabs(B[(int64_t)i * ldb + j]);
    m = fmax(m, s);
  }
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sm[0];
}

template <class T>
void small_inf_norm(apf_ctx* ctx, int64_t p, const T* B, int64_t ldb, double* out) {
  k_inf_norm<T><<<1, 256, 0, ctx->stream>>>((int)p, B, ldb, out);
  count_launch(ctx);
}
template void small_inf_norm<double>(apf_ctx*, int64_t, const double*, int64_t, double*);
template void small_inf_norm<double2>(apf_ctx*, int64_t, const double2*, int64_t, double*);

// ---- one-sided Jacobi ---------------------------------------------------------------
// M (column-major, ld = p) = B + s I with s = 2 ||B||_inf (1 if B = 0)
template <class T>
__global__ void k_shifted_colmajor(int p, const T* __restrict__ B, int64_t ldb,
                                   const double* __restrict__ nrm, T* __restrict__ M) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)p * p) return;
  const int j = (int)(e / p), i = (int)(e % p);
  double s = 2.0 * nrm[0];
  if (!(s > 0.0)) s = 1.0;
  T v = B[(int64_t)i * ldb + j];
  if (i == j) v = add(v, make_val<T>(s, 0.0));
  M[(int64_t)j * p + i] = v;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier for a cooperative launch.  bar[0]: arrivals, bar[1]: generation.
// Returns false (and records DEV_BARRIER_TIMEOUT) if the other blocks do not
// arrive within the time limit; callers then leave the kernel.
__device__ bool grid_barrier(unsigned* bar, unsigned& gen, unsigned nblocks, int* err, uint64_t limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    const unsigned prev = atomicAdd(&bar[0], 1u);
    if (prev == nblocks - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (atomicAdd(&bar[1], 0u) == gen) {
        __nanosleep(64);
        if (global_ns() - t0 > limit_ns) {  // 2 s unless the context sets another limit
          set_err(err, DEV_BARRIER_TIMEOUT);
          ok = 0;
          break;
        }
        if (*(volatile int*)err == DEV_BARRIER_TIMEOUT) { ok = 0; break; }
      }
    }
    __threadfence();
  }
  ++gen;
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ int rr_index(int pos, int r, int P) {
  return pos == 0 ? 0 : 1 + (pos - 1 + r) % (P - 1);
}

template <class T>
__global__ void __launch_bounds__(128) k_jacobi_sweeps(int p, int P, T* M, unsigned* bar,
                                                       unsigned* counters, int max_sweeps,
                                                       double tol, int* err, uint64_t limit_ns) {
  const int lane = threadIdx.x % 32;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int nw = gridDim.x * blockDim.x / 32;
  unsigned gen = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < P - 1; ++r) {
      for (int pr = gw; pr < P / 2; pr += nw) {
        const int ia = rr_index(pr, r, P), ib = rr_index(P - 1 - pr, r, P);
        if (ia >= p || ib >= p) continue;
        T* ma = M + (int64_t)ia * p;
        T* mb = M + (int64_t)ib * p;
        double al = 0.0, be = 0.0;
        T ga = szero<T>();
        for (int i = lane; i < p; i += 32) {
          const T x = ma[i], y = mb[i];
          al += abs2(x);
          be += abs2(y);
          madd_conj(ga, x, y);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        const double g = rabs(ga);
        if (g > tol * sqrt(al * be) && g > 0.0) {
          const double zeta = (be - al) / (2.0 * g);
          double t;
          if (fabs(zeta) > 1e100) t = 0.5 / zeta;
          else t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          const T ph = rmul(1.0 / g, ga);       // e^{i phi} = gamma / |gamma|
          const T sp = rmul(s, ph);             // s e^{i phi}
          const T spc = conj_(sp);              // s e^{-i phi}
          for (int i = lane; i < p; i += 32) {
            const T x = ma[i], y = mb[i];
            ma[i] = sub(rmul(c, x), mul(spc, y));
            mb[i] = add(mul(sp, x), rmul(c, y));
          }
          if (lane == 0) atomicAdd(&counters[sweep], 1u);
        }
      }
      if (!grid_barrier(bar, gen, gridDim.x, err, limit_ns)) return;
    }
    if (atomicAdd(&counters[sweep], 0u) == 0u) return;  // a sweep without rotations
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) set_err(err, DEV_EIGH_NOCONV);
}

// column j: sigma_j = ||m_j||, u_j = m_j / sigma_j, lambda_j = u_j^H B u_j
template <class T>
__global__ void k_jacobi_finish(int p, T* M, const T* __restrict__ B, int64_t ldb,
                                double* __restrict__ lam) {
  const int j = blockIdx.x;
  T* m = M + (int64_t)j * p;
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) s += abs2(m[i]);
  s = warp_sum(s);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const double inv = 1.0 / sqrt(red[0]);
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += blockDim.x) m[i] = rmul(inv, m[i]);
  __syncthreads();
  // Rayleigh quotient: sum_i conj(u_i) sum_k B_ik u_k
  double q = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    T bu = szero<T>();
    for (int k = 0; k < p; ++k) madd(bu, B[(int64_t)i * ldb + k], m[k]);
    T t = szero<T>();
    madd_conj(t, m[i], bu);
    q += real_(t);
  }
  q = warp_sum(q);
  __syncthreads();
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = q;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) lam[j] = v;
  }
}

// sort ascending (ties by index); w[rank_j] = lam_j, U[:, rank_j] = u_j (row-major U)
template <class T>
__global__ void k_jacobi_sort(int p, const double* __restrict__ lam, const T* __restrict__ M,
                              double* __restrict__ w, T* __restrict__ U, int64_t ldu) {
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const double lj = lam[j];
    int rank = 0;
    for (int i = 0; i < p; ++i) {
      const double li = lam[i];
      rank += (li < lj) || (li == lj && i < j);
    }
    w[rank] = lj;
    for (int i = 0; i < p; ++i) U[(int64_t)i * ldu + rank] = M[(int64_t)j * p + i];
  }
}

template <class T>
void eigh_jacobi(apf_ctx* ctx, int64_t p, const T* B, int64_t ldb, double* w, T* U, int64_t ldu) {
  if (p == 0) return;
  APF_REQUIRE(p <= APF_MAX_P, APF_ERR_ARG);
  const int P = (int)(p + (p & 1));
  DBuf Mb((size_t)p * p * sizeof(T) + 64, ctx->stream, false);
  DBuf scal(sizeof(double) * (size_t)(p + 2), ctx->stream, false);
  T* M = Mb.as<T>();
  double* nrm = scal.as<double>();
  double* lam = nrm + 2;
  small_inf_norm<T>(ctx, p, B, ldb, nrm);
  k_shifted_colmajor<T><<<(unsigned)((p * p + 255) / 256), 256, 0, ctx->stream>>>((int)p, B, ldb, nrm, M);
  count_launch(ctx);
  const int max_sweeps = 40;
  APF_CUDA(cudaMemsetAsync(ctx->d_bar, 0, 2 * sizeof(unsigned), ctx->stream));
  APF_CUDA(cudaMemsetAsync(ctx->d_counters, 0, 64 * sizeof(unsigned), ctx->stream));
  const int threads = 128;
  int per_sm = 0;
  APF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_sweeps<T>, threads, 0));
  int nb = (P / 2 + (threads / 32) - 1) / (threads / 32);
  const int cap = per_sm * ctx->num_sms;
  if (nb > cap) nb = cap;
  if (nb > ctx->num_sms) nb = ctx->num_sms;
  if (nb < 1) nb = 1;
  int pi = (int)p;
  double tol = (double)p * 2.220446049250313e-16;
  unsigned* bar = ctx->d_bar;
  unsigned* counters = ctx->d_counters;
  int* err = ctx->d_err;
  int ms = max_sweeps;
  int Pv = P;
  uint64_t limit = barrier_wait_ns(ctx);
  void* args[] = {&pi, &Pv, &M, &bar, &counters, &ms, &tol, &err, &limit};
  APF_CUDA(cudaLaunchCooperativeKernel((void*)k_jacobi_sweeps<T>, dim3(nb), dim3(threads), args, 0,
                                       ctx->stream));
  k_jacobi_finish<T><<<(unsigned)p, 128, 0, ctx->stream>>>((int)p, M, B, ldb, lam);
  k_jacobi_sort<T><<<1, 1024, 0, ctx->stream>>>((int)p, lam, M, w, U, ldu);
  count_launch(ctx, 3);
}
// Failure-path check of the eigensolver's grid barrier: the blocks of a
// cooperative launch wait for one more arrival than there are blocks, which
// never comes; each gives up after the context's wait limit.
__global__ void k_barrier_probe(unsigned* bar, int* err, uint64_t limit_ns) {
  unsigned gen = 0;
  grid_barrier(bar, gen, gridDim.x + 1, err, limit_ns);
}

void wait_probe_barrier(apf_ctx* ctx) {
  APF_CUDA(cudaMemsetAsync(ctx->d_bar, 0, 2 * sizeof(unsigned), ctx->stream));
  unsigned* bar = ctx->d_bar;
  int* err = ctx->d_err;
  uint64_t limit = barrier_wait_ns(ctx);
  void* args[] = {&bar, &err, &limit};
  APF_CUDA(cudaLaunchCooperativeKernel((void*)k_barrier_probe, dim3(2), dim3(128), args, 0, ctx->stream));
  count_launch(ctx);
  APF_CUDA(cudaMemsetAsync(ctx->d_bar, 0, 2 * sizeof(unsigned), ctx->stream));
  const int e = fetch_device_error(ctx);
  if (e == DEV_BARRIER_TIMEOUT) throw ApfError{APF_ERR_TIMEOUT, "eigensolver grid barrier"};
  if (e != 0) throw ApfError{APF_ERR_CUDA, "device error in the wait probe"};
}

template void eigh_jacobi<double>(apf_ctx*, int64_t, const double*, int64_t, double*, double*, int64_t);
template void eigh_jacobi<double2>(apf_ctx*, int64_t, const double2*, int64_t, double*, double2*,
                                   int64_t);

}  // namespace apf
