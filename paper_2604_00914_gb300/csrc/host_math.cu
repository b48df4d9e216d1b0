// Scalar set-up of the filter, computed once per solve on the host in FP64
// (O(k) and O(p k) work between device phases):
//  - step-function Chebyshev coefficients c_j (Sec. 2.2, Eq. (c_j));
//  - damping factors: exponent-m Lanczos (Eq. (m_Lanczos_damping)) or Jackson;
//  - initial degree k^(1) (Eq. (compute_k_1)) and maximum degree k (Sec. 4);
//  - the degree of the next iteration (Alg. 3).
#include <math.h>

#include <algorithm>
#include <vector>

#include "apf_internal.h"
#include "host_math.h"

namespace apf {

static const double kPi = 3.14159265358979323846;

std::vector<double> filter_coefficients(double am, double bm, int k, int damping, double m) {
  std::vector<double> a((size_t)k + 1);
  const double al = acos(am), be = acos(bm);
  for (int j = 0; j <= k; ++j) {
    double c;
    if (j == 0) c = (al - be) / kPi;
    else c = 2.0 / kPi * (sin(j * al) - sin(j * be)) / j;
    double d = 1.0;
    if (damping == APF_DAMP_LANCZOS_M && j > 0) {
      const double u = j * kPi / (k + 1);
      d = pow(sin(u) / u, m);
    } else if (damping == APF_DAMP_JACKSON) {
      const double t = kPi / (k + 2);
      d = ((k + 2 - j) * sin(t) * cos(j * t) + cos(t) * sin(j * t)) / ((k + 2) * sin(t));
    }
    a[(size_t)j] = c * d;
  }
  return a;
}

int initial_degree(double am, double bm, double C) {
  return (int)ceil(C / (acos(am) - acos(bm))) - 1;
}

int degree_select(const double* ritz, int p, int e, const double* a, int k, double l1, double l2,
                  double tau_a) {
  if (e < 1 || e > p) return k;
  std::vector<double> x((size_t)p), t0((size_t)p, 1.0), t1((size_t)p), g((size_t)p), mag((size_t)p);
  for (int c = 0; c < p; ++c) {
    x[(size_t)c] = l1 * ritz[c] + l2;
    t1[(size_t)c] = x[(size_t)c];
    g[(size_t)c] = a[0];
  }
  for (int j = 1; j <= k; ++j) {
    for (int c = 0; c < p; ++c) {
      g[(size_t)c] += a[j] * t1[(size_t)c];
      mag[(size_t)c] = fabs(g[(size_t)c]);
    }
    // the p-th and e-th largest magnitudes
    std::vector<double> srt(mag);
    std::sort(srt.begin(), srt.end(), [](double u, double v) { return u > v; });
    if (srt[(size_t)p - 1] < tau_a * srt[(size_t)e - 1]) return j;
    for (int c = 0; c < p; ++c) {
      const double tn = 2.0 * x[(size_t)c] * t1[(size_t)c] - t0[(size_t)c];
      t0[(size_t)c] = t1[(size_t)c];
      t1[(size_t)c] = tn;
    }
  }
  return k;
}

}  // namespace apf
