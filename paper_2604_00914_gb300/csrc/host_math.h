#pragma once
#include <vector>

namespace apf {
// a_j = c_j d_{j,k}, j = 0..k for the mapped interval [am, bm]
std::vector<double> filter_coefficients(double am, double bm, int k, int damping, double m);
// k^(1) = ceil(C / (arccos am - arccos bm)) - 1
int initial_degree(double am, double bm, double C);
// Alg. 3
int degree_select(const double* ritz, int p, int e, const double* a, int k, double l1, double l2,
                  double tau_a);
}  // namespace apf
