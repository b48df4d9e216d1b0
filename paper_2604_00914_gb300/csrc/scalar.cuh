// Real and complex scalar helpers shared by the kernels.
//
// Storage types: double, double2 (complex FP64), float, float2 (complex FP32).
// Complex values are (x = re, y = im).  Each helper is written for all four.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace apf {

template <class T> struct ScalarTraits;
template <> struct ScalarTraits<double> {
  using Real = double;
  static constexpr bool is_complex = false;
  static constexpr int per16 = 2;  // elements per 16-byte vector
};
template <> struct ScalarTraits<double2> {
  using Real = double;
  static constexpr bool is_complex = true;
  static constexpr int per16 = 1;
};
template <> struct ScalarTraits<float> {
  using Real = float;
  static constexpr bool is_complex = false;
  static constexpr int per16 = 4;
};
template <> struct ScalarTraits<float2> {
  using Real = float;
  static constexpr bool is_complex = true;
  static constexpr int per16 = 2;
};

__host__ __device__ __forceinline__ double zero_of(double) { return 0.0; }
__host__ __device__ __forceinline__ float zero_of(float) { return 0.0f; }
__host__ __device__ __forceinline__ double2 zero_of(double2) { return make_double2(0.0, 0.0); }
__host__ __device__ __forceinline__ float2 zero_of(float2) { return make_float2(0.0f, 0.0f); }

template <class T> __host__ __device__ __forceinline__ T szero() { return zero_of(T()); }

// a + b
__host__ __device__ __forceinline__ double add(double a, double b) { return a + b; }
__host__ __device__ __forceinline__ float add(float a, float b) { return a + b; }
__host__ __device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
// a - b
__host__ __device__ __forceinline__ double sub(double a, double b) { return a - b; }
__host__ __device__ __forceinline__ float sub(float a, float b) { return a - b; }
__host__ __device__ __forceinline__ double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * b
__host__ __device__ __forceinline__ double mul(double a, double b) { return a * b; }
__host__ __device__ __forceinline__ float mul(float a, float b) { return a * b; }
__host__ __device__ __forceinline__ double2 mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// real scalar times value
__host__ __device__ __forceinline__ double rmul(double s, double a) { return s * a; }
__host__ __device__ __forceinline__ float rmul(float s, float a) { return s * a; }
__host__ __device__ __forceinline__ double2 rmul(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 rmul(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
// conj
__host__ __device__ __forceinline__ double conj_(double a) { return a; }
__host__ __device__ __forceinline__ float conj_(float a) { return a; }
__host__ __device__ __forceinline__ double2 conj_(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 conj_(float2 a) { return make_float2(a.x, -a.y); }
// acc += a * b   (fused multiply-adds)
__host__ __device__ __forceinline__ void madd(double& acc, double a, double b) { acc = fma(a, b, acc); }
__host__ __device__ __forceinline__ void madd(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__host__ __device__ __forceinline__ void madd(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ void madd(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__host__ __device__ __forceinline__ void madd_conj(double& acc, double a, double b) { acc = fma(a, b, acc); }
__host__ __device__ __forceinline__ void madd_conj(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// One output of a Clenshaw step, alpha acc - v + f y (terms without Vin or Y
// dropped), with every rounding fixed by explicit round-to-nearest operations
// so that no kernel variant depends on the compiler's choice of fusions:
// r = fma(alpha, acc, -v) (or alpha acc, exact for alpha = 1, 2), then
// r = fma(f, y, r).  Complex values: the same on each component.
template <class R>
__device__ __forceinline__ R fma_rn(R a, R b, R c);
template <> __device__ __forceinline__ float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <class R>
__device__ __forceinline__ R mul_rn(R a, R b);
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <class R>
__device__ __forceinline__ R step_comp(R acc, R alpha, bool hv, R v, bool hy, R f, R y) {
  const R r = hv ? fma_rn<R>(alpha, acc, -v) : mul_rn<R>(alpha, acc);
  return hy ? fma_rn<R>(f, y, r) : r;
}
__device__ __forceinline__ float step_out(float acc, float al, bool hv, float v, bool hy, float f, float y) {
  return step_comp<float>(acc, al, hv, v, hy, f, y);
}
__device__ __forceinline__ double step_out(double acc, double al, bool hv, double v, bool hy, double f, double y) {
  return step_comp<double>(acc, al, hv, v, hy, f, y);
}
__device__ __forceinline__ float2 step_out(float2 acc, float al, bool hv, float2 v, bool hy, float f, float2 y) {
  return make_float2(step_comp<float>(acc.x, al, hv, v.x, hy, f, y.x), step_comp<float>(acc.y, al, hv, v.y, hy, f, y.y));
}
__device__ __forceinline__ double2 step_out(double2 acc, double al, bool hv, double2 v, bool hy, double f, double2 y) {
  return make_double2(step_comp<double>(acc.x, al, hv, v.x, hy, f, y.x),
                      step_comp<double>(acc.y, al, hv, v.y, hy, f, y.y));
}

// |a|^2
__host__ __device__ __forceinline__ double abs2(double a) { return a * a; }
__host__ __device__ __forceinline__ double abs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float abs2(float a) { return a * a; }
__host__ __device__ __forceinline__ float abs2(float2 a) { return a.x * a.x + a.y * a.y; }
// Re(conj(a) b)
__host__ __device__ __forceinline__ double re_dot(double a, double b) { return a * b; }
__host__ __device__ __forceinline__ double re_dot(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }
// real part
__host__ __device__ __forceinline__ double real_(double a) { return a; }
__host__ __device__ __forceinline__ double real_(double2 a) { return a.x; }

// conversions between precisions
__host__ __device__ __forceinline__ float to_lo(double a) { return (float)a; }
__host__ __device__ __forceinline__ float2 to_lo(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double to_hi(float a) { return (double)a; }
__host__ __device__ __forceinline__ double2 to_hi(float2 a) { return make_double2((double)a.x, (double)a.y); }

template <class T> struct LowOf;
template <> struct LowOf<double> { using type = float; };
template <> struct LowOf<double2> { using type = float2; };

// make a value from (re, im); imaginary part dropped for real types
template <class T> __host__ __device__ __forceinline__ T make_val(double re, double im);
template <> __host__ __device__ __forceinline__ double make_val<double>(double re, double) { return re; }
template <> __host__ __device__ __forceinline__ double2 make_val<double2>(double re, double im) { return make_double2(re, im); }
template <> __host__ __device__ __forceinline__ float make_val<float>(double re, double) { return (float)re; }
template <> __host__ __device__ __forceinline__ float2 make_val<float2>(double re, double im) { return make_float2((float)re, (float)im); }

// warp shuffles of scalar types
__device__ __forceinline__ double shfl(double v, int src, int width) { return __shfl_sync(0xffffffffu, v, src, width); }
__device__ __forceinline__ float shfl(float v, int src, int width) { return __shfl_sync(0xffffffffu, v, src, width); }
__device__ __forceinline__ double2 shfl(double2 v, int src, int width) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src, width), __shfl_sync(0xffffffffu, v.y, src, width));
}
__device__ __forceinline__ float2 shfl(float2 v, int src, int width) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src, width), __shfl_sync(0xffffffffu, v.y, src, width));
}
__device__ __forceinline__ double shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double2 shfl_xor(double2 v, int m) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = add(v, shfl_xor(v, m));
  return v;
}

}  // namespace apf
