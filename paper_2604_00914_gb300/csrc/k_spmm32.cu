// FP32 instantiations of the Clenshaw step (real and complex), the filter
// recurrence of APF_FILTER_F32 / APF_FILTER_F32_DEFECT.
#include "spmm_impl.cuh"

namespace apf {

template <class T, class TA>
void clenshaw_step(apf_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* colidx,
                   const TA* vals, const T* W, const T* Vin, const T* Y, int64_t ld,
                   int64_t ncols, const typename ScalarTraits<T>::Real* coef_col,
                   typename ScalarTraits<T>::Real coef_scalar,
                   typename ScalarTraits<T>::Real alpha, T* Out) {
  clenshaw_step_impl<T, TA>(ctx, n, rowptr, colidx, vals, W, Vin, Y, ld, ncols, coef_col,
                            coef_scalar, alpha, Out);
}

template void clenshaw_step<float, float>(apf_ctx*, int64_t, const int64_t*, const int32_t*,
                                          const float*, const float*, const float*, const float*,
                                          int64_t, int64_t, const float*, float, float, float*);
template void clenshaw_step<float2, float2>(apf_ctx*, int64_t, const int64_t*, const int32_t*,
                                            const float2*, const float2*, const float2*,
                                            const float2*, int64_t, int64_t, const float*, float,
                                            float, float2*);

}  // namespace apf
