// The AdaPolySI driver (Alg. 4) and the step functions exposed through the C ABI.
#pragma once
#include <vector>

#include "apf_internal.h"

struct apf_result {
  apf_ctx* ctx = nullptr;
  int64_t n = 0, e = 0;
  int dtype = APF_R64;
  apf::DBuf vecs;                 // n x lde row-major eigenvectors
  int64_t lde = 0;
  std::vector<double> lam, res;   // ascending eigenvalues, relative residuals
  std::vector<double> history;    // 6 doubles per iteration
  std::vector<int64_t> slice_counts;  // per slice, input order (apf_solve_slices)
  apf_stats stats{};
  bool owns_ctx = false;  // a serving request's result: destroying it destroys its context
};

namespace apf {

void solve(apf_ctx* ctx, const apf_matrix* A, const apf_params* prm, apf_result* out);
void solve_slices(apf_ctx* ctx, const apf_matrix* A, int nslices, const double* a, const double* b,
                  const int64_t* p, const apf_params* prm, apf_result* out);

// Alg. 2 on caller blocks (FP64 input/output of the matrix dtype)
template <class T>
void filter_apply_public(apf_ctx* ctx, const apf_matrix* A, const double* coef, int k, double l1,
                         double l2, int precision, const T* X, int64_t ldx, int64_t p, T* Y,
                         int64_t ldy);
template <class T>
void filter_apply_defect_public(apf_ctx* ctx, const apf_matrix* A, const double* coef, int k,
                                double l1, double l2, const T* V, const T* AV, const double* lam,
                                int64_t ld, int64_t p, T* Y, int64_t ldy);
template <class T>
double count_estimate_public(apf_ctx* ctx, const apf_matrix* A, const double* coef, int k, double l1, double l2,
                             int precision, int64_t m, uint64_t seed);
template <class T>
void spmm_public(apf_ctx* ctx, const apf_matrix* A, const T* X, int64_t ldx, int64_t p, T* Y,
                 int64_t ldy);
template <class T>
void cholqr2_public(apf_ctx* ctx, int64_t n, int64_t p, T* X, int64_t ld);
template <class T>
void rayleigh_ritz_public(apf_ctx* ctx, const apf_matrix* A, const T* Q, int64_t ld, int64_t p,
                          double* w, T* V, int64_t ldv);
// failure-path checks: kernels whose device-side wait nothing satisfies
void wait_probe_pair(apf_ctx* ctx, const apf_matrix* A);
void wait_probe_barrier(apf_ctx* ctx);

template <class T>
void residual_norms_public(apf_ctx* ctx, const apf_matrix* A, const T* V, int64_t ld, int64_t p,
                           const double* w, double* host_out);

}  // namespace apf
