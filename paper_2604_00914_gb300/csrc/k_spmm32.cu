// FP32 instantiations of the Clenshaw step (real and complex), the filter
// recurrence of APF_FILTER_F32 / APF_FILTER_F32_DEFECT: the CSR kernel, the
// SELL-8 kernel with TMA bulk staging, and the SELL value gather.
#include "spmm_sell_ct.cuh"

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

template <class T, class TA>
void clenshaw_step_shape(apf_ctx* ctx, int G, int VPT, int64_t n, const int64_t* rowptr,
                         const int32_t* colidx, const TA* vals, const T* W, const T* Vin, const T* Y,
                         int64_t ld, int64_t ncols, const typename ScalarTraits<T>::Real* coef_col,
                         typename ScalarTraits<T>::Real coef_scalar,
                         typename ScalarTraits<T>::Real alpha, T* Out) {
  clenshaw_step_impl<T, TA>(ctx, G, VPT, n, rowptr, colidx, vals, W, Vin, Y, ld, ncols, coef_col,
                            coef_scalar, alpha, Out);
}

template <class T, class TA>
void clenshaw_step_sell(apf_ctx* ctx, int G, int VPT, int64_t n, const int64_t* chunk_ptr,
                        const int32_t* scol, const TA* sval, int lmax, const T* W, const T* Vin,
                        const T* Y, int64_t ld, int64_t ncols,
                        const typename ScalarTraits<T>::Real* coef_col,
                        typename ScalarTraits<T>::Real coef_scalar,
                        typename ScalarTraits<T>::Real alpha, T* Out) {
  clenshaw_sell_launch<T, TA>(ctx, G, VPT, n, chunk_ptr, scol, sval, lmax, W, Vin, Y, ld, ncols,
                              coef_col, coef_scalar, alpha, Out);
}

template <class T, class TA>
void clenshaw_sell_pair(apf_ctx* ctx, int G, int VPT, int64_t n, const int64_t* chunk_ptr,
                        const int32_t* scol, const TA* sval, int lmax, int64_t bandwidth, T* bufA,
                        T* bufB, const T* va, const T* Y, int64_t ld, int64_t ncols,
                        const typename ScalarTraits<T>::Real* coef1_col,
                        typename ScalarTraits<T>::Real coef1,
                        const typename ScalarTraits<T>::Real* coef2_col,
                        typename ScalarTraits<T>::Real coef2, unsigned* seg_count, unsigned pass) {
  clenshaw_sell_pair_launch<T, TA>(ctx, G, VPT, n, chunk_ptr, scol, sval, lmax, bandwidth, bufA, bufB, va, Y,
                                   ld, ncols, coef1_col, coef1, coef2_col, coef2, seg_count, pass);
}

template <class T, class TA>
void clenshaw_step_sell_ct(apf_ctx* ctx, int G, int VPT, int64_t n, const int64_t* chunk_ptr,
                           const int32_t* scol, const TA* sval, int lmax, const T* W, const T* Vin,
                           const T* Y, int64_t ld, int64_t ncols,
                           const typename ScalarTraits<T>::Real* coef_col,
                           typename ScalarTraits<T>::Real coef_scalar,
                           typename ScalarTraits<T>::Real alpha, T* Out, int halo) {
  clenshaw_sell_ct_launch<T, TA>(ctx, G, VPT, n, chunk_ptr, scol, sval, lmax, W, Vin, Y, ld, ncols, coef_col,
                                 coef_scalar, alpha, Out, halo);
}

template <class TA>
__global__ void k_sell_gather(int64_t slots, const int32_t* __restrict__ src, const TA* __restrict__ csr,
                              TA* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= slots) return;
  const int32_t e = src[s];
  out[s] = e >= 0 ? csr[e] : szero<TA>();
}

template <class TA>
void sell_gather_values(apf_ctx* ctx, int64_t slots, const int32_t* src, const TA* csr, TA* out) {
  if (slots == 0) return;
  k_sell_gather<TA><<<(unsigned)((slots + 255) / 256), 256, 0, ctx->stream>>>(slots, src, csr, out);
  count_launch(ctx);
}

#define APF_INST32(T)                                                                                 \
  template void clenshaw_step<T, T>(apf_ctx*, int64_t, const int64_t*, const int32_t*, const T*,      \
                                    const T*, const T*, const T*, int64_t, int64_t, const float*,     \
                                    float, float, T*);                                                \
  template void clenshaw_step_shape<T, T>(apf_ctx*, int, int, int64_t, const int64_t*,                \
                                          const int32_t*, const T*, const T*, const T*, const T*,     \
                                          int64_t, int64_t, const float*, float, float, T*);          \
  template void clenshaw_step_sell<T, T>(apf_ctx*, int, int, int64_t, const int64_t*, const int32_t*, \
                                         const T*, int, const T*, const T*, const T*, int64_t,        \
                                         int64_t, const float*, float, float, T*);                    \
  template void clenshaw_step_sell_ct<T, T>(apf_ctx*, int, int, int64_t, const int64_t*, const int32_t*, \
                                            const T*, int, const T*, const T*, const T*, int64_t,        \
                                            int64_t, const float*, float, float, T*, int);               \
  template void sell_gather_values<T>(apf_ctx*, int64_t, const int32_t*, const T*, T*);              \
  template void clenshaw_sell_pair<T, T>(apf_ctx*, int, int, int64_t, const int64_t*, const int32_t*, \
                                         const T*, int, int64_t, T*, T*, const T*, const T*, int64_t, \
                                         int64_t, const float*, float, const float*, float, unsigned*, \
                                         unsigned);
APF_INST32(float)
APF_INST32(float2)
#undef APF_INST32

}  // namespace apf
