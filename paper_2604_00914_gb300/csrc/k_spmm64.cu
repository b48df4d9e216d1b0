// FP64 instantiations of the Clenshaw step, plus the other sparse kernels:
// single-vector SpMV (Lanczos), the shifted/scaled copy of A used by the
// filter (A_hat = l1 A + l2 I), and the Gershgorin interval.
#include "spmm_impl.cuh"

namespace apf {

template <class T, class TA>
void clenshaw_step(apf_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* colidx,
                   const TA* vals, const T* W, const T* Vin, const T* Y, int64_t ld,
                   int64_t ncols, const typename ScalarTraits<T>::Real* coef_col,
                   typename ScalarTraits<T>::Real coef_scalar,
                   typename ScalarTraits<T>::Real alpha, T* Out) {
  clenshaw_step_impl<T, TA>(ctx, 0, 0, n, rowptr, colidx, vals, W, Vin, Y, ld, ncols, coef_col,
                            coef_scalar, alpha, Out);
}

template void clenshaw_step<double, double>(apf_ctx*, int64_t, const int64_t*, const int32_t*,
                                            const double*, const double*, const double*,
                                            const double*, int64_t, int64_t, const double*, double,
                                            double, double*);
template void clenshaw_step<double2, double2>(apf_ctx*, int64_t, const int64_t*, const int32_t*,
                                              const double2*, const double2*, const double2*,
                                              const double2*, int64_t, int64_t, const double*,
                                              double, double, double2*);

// ---- single-vector SpMV: y = A x, one thread per row -------------------------
template <class T>
__global__ void k_spmv(int64_t n, const int64_t* __restrict__ rowptr,
                       const int32_t* __restrict__ colidx, const T* __restrict__ vals,
                       const T* __restrict__ x, T* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T acc = szero<T>();
  for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) madd(acc, vals[e], x[colidx[e]]);
  y[i] = acc;
}

template <class T>
void spmv(apf_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* colidx, const T* vals,
          const T* x, T* y) {
  if (n == 0) return;
  k_spmv<T><<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, rowptr, colidx, vals, x, y);
  count_launch(ctx);
}
template void spmv<double>(apf_ctx*, int64_t, const int64_t*, const int32_t*, const double*,
                           const double*, double*);
template void spmv<double2>(apf_ctx*, int64_t, const int64_t*, const int32_t*, const double2*,
                            const double2*, double2*);

// ---- A_hat = l1 A + l2 I, rounded to the output precision ----------------------
template <class T, class TO>
__global__ void k_scale_shift(int64_t n, const int64_t* __restrict__ rowptr,
                              const int32_t* __restrict__ colidx, const T* __restrict__ vals,
                              double l1, double l2, TO* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    T v = rmul(l1, vals[e]);
    if (colidx[e] == i) v = add(v, make_val<T>(l2, 0.0));
    if constexpr (sizeof(TO) == sizeof(T)) {
      out[e] = v;
    } else {
      out[e] = to_lo(v);
    }
  }
}

template <class T, class TO>
void scale_shift_matrix(apf_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* colidx,
                        const T* vals, double l1, double l2, TO* out) {
  if (n == 0) return;
  k_scale_shift<T, TO><<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, rowptr, colidx,
                                                                             vals, l1, l2, out);
  count_launch(ctx);
}
template void scale_shift_matrix<double, double>(apf_ctx*, int64_t, const int64_t*, const int32_t*,
                                                 const double*, double, double, double*);
template void scale_shift_matrix<double, float>(apf_ctx*, int64_t, const int64_t*, const int32_t*,
                                                const double*, double, double, float*);
template void scale_shift_matrix<double2, double2>(apf_ctx*, int64_t, const int64_t*,
                                                   const int32_t*, const double2*, double, double,
                                                   double2*);
template void scale_shift_matrix<double2, float2>(apf_ctx*, int64_t, const int64_t*,
                                                  const int32_t*, const double2*, double, double,
                                                  float2*);

// ---- Gershgorin interval: per-block min/max, then one block reduces ------------
__device__ __forceinline__ double abs_(double v) { return fabs(v); }
__device__ __forceinline__ double abs_(double2 v) { return hypot(v.x, v.y); }

template <class T>
__global__ void k_gersh_partial(int64_t n, const int64_t* __restrict__ rowptr,
                                const int32_t* __restrict__ colidx, const T* __restrict__ vals,
                                double* __restrict__ part) {
  __shared__ double slo[256], shi[256];
  double lo = 1e300, hi = -1e300;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double c = 0.0, r = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      if (colidx[e] == i) c = real_(vals[e]);
      else r += abs_(vals[e]);
    }
    lo = fmin(lo, c - r);
    hi = fmax(hi, c + r);
  }
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + s]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = slo[0];
    part[2 * blockIdx.x + 1] = shi[0];
  }
}

__global__ void k_minmax_final(int nb, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double slo[256], shi[256];
  double lo = 1e300, hi = -1e300;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    lo = fmin(lo, part[2 * b]);
    hi = fmax(hi, part[2 * b + 1]);
  }
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + s]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = slo[0];
    out[1] = shi[0];
  }
}

template <class T>
void gershgorin(apf_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* colidx,
                const T* vals, double* lo, double* hi) {
  int nb = (int)((n + 255) / 256);
  if (nb > 4 * ctx->num_sms) nb = 4 * ctx->num_sms;
  if (nb < 1) nb = 1;
  DBuf part((size_t)nb * 2 * sizeof(double) + 2 * sizeof(double), ctx->stream, false);
  double* p = part.as<double>();
  k_gersh_partial<T><<<nb, 256, 0, ctx->stream>>>(n, rowptr, colidx, vals, p);
  k_minmax_final<<<1, 256, 0, ctx->stream>>>(nb, p, p + 2 * nb);
  count_launch(ctx, 2);
  double h[2];
  APF_CUDA(cudaMemcpyAsync(h, p + 2 * nb, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  APF_CUDA(cudaStreamSynchronize(ctx->stream));
  *lo = h[0];
  *hi = h[1];
}
template void gershgorin<double>(apf_ctx*, int64_t, const int64_t*, const int32_t*, const double*,
                                 double*, double*);
template void gershgorin<double2>(apf_ctx*, int64_t, const int64_t*, const int32_t*,
                                  const double2*, double*, double*);

}  // namespace apf
