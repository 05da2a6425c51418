// The elliptical NFW halo of the composite mass class as a sum of cored steep ellipsoids
// (App. B: the eNFW convergence kappa_s k(xi / r_s) written as 44 CSEs).  The paper takes the
// decomposition from the literature without printing it; here it is fitted once per process:
// cores s_i log-spaced on [1e-5, 1e4] (units of r_s) and amplitudes a_i >= 0 minimising the
// relative error of sum_i a_i (u^2 + s_i^2)^(-3/2) against the projected NFW shape
//   k(u) = 2 (1 - F(u)) / (u^2 - 1),  F = arctanh(sqrt(1 - u^2)) / sqrt(1 - u^2)  (u < 1),
//                                         arctan(sqrt(u^2 - 1)) / sqrt(u^2 - 1)    (u > 1),
// on 2000 points log-spaced over u in [1e-4, 1e3], by non-negative least squares (the active-set
// method of Lawson & Hanson, with Householder QR for each passive-set subproblem).
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "glad_internal.cuh"

namespace {

// projected NFW shape k(u), u > 0; near u = 1 the series 2 sum_n w^(2n) / (2n + 3), w^2 = 1 - u^2
double nfw_shape(double u) {
  const double w2 = 1.0 - u * u;
  if (fabs(w2) < 1e-2) {
    double s = 0.0, p = 1.0;
    for (int n = 0; n < 12; ++n, p *= w2) s += 2.0 * p / (2 * n + 3);
    return s;
  }
  double F;
  if (u < 1.0) {
    const double w = sqrt(w2);
    F = atanh(w) / w;
  } else {
    const double w = sqrt(-w2);
    F = atan(w) / w;
  }
  return 2.0 * (1.0 - F) / (u * u - 1.0);
}

// min ||A z - b||_2 over the columns `cols` of A (m x n, column-major) by Householder QR.
void ls_subset(const std::vector<double> &A, int m, const std::vector<int> &cols,
               const std::vector<double> &b, std::vector<double> &z) {
  const int k = (int)cols.size();
  std::vector<double> Q((size_t)m * k), r = b;
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < m; ++i) Q[(size_t)j * m + i] = A[(size_t)cols[j] * m + i];
  for (int j = 0; j < k; ++j) {
    double *v = &Q[(size_t)j * m];
    double nrm = 0.0;
    for (int i = j; i < m; ++i) nrm += v[i] * v[i];
    nrm = sqrt(nrm);
    if (nrm == 0.0) continue;
    const double alpha = v[j] > 0 ? -nrm : nrm;
    // reflector u = v - alpha e_j (stored in v[j..m)), applied to the later columns and to r
    v[j] -= alpha;
    double uu = 0.0;
    for (int i = j; i < m; ++i) uu += v[i] * v[i];
    for (int c = j + 1; c < k; ++c) {
      double *w = &Q[(size_t)c * m];
      double d = 0.0;
      for (int i = j; i < m; ++i) d += v[i] * w[i];
      d = 2.0 * d / uu;
      for (int i = j; i < m; ++i) w[i] -= d * v[i];
    }
    double d = 0.0;
    for (int i = j; i < m; ++i) d += v[i] * r[i];
    d = 2.0 * d / uu;
    for (int i = j; i < m; ++i) r[i] -= d * v[i];
    // the diagonal of R is alpha; keep it where back-substitution reads it
    v[j] = alpha;
  }
  z.assign(k, 0.0);
  for (int j = k - 1; j >= 0; --j) {
    double s = r[j];
    for (int c = j + 1; c < k; ++c) s -= Q[(size_t)c * m + j] * z[c];
    const double d = Q[(size_t)j * m + j];
    z[j] = d != 0.0 ? s / d : 0.0;
  }
}

// Lawson & Hanson non-negative least squares: min ||A x - b|| subject to x >= 0.
void nnls(const std::vector<double> &A, int m, int n, const std::vector<double> &b,
          std::vector<double> &x) {
  x.assign(n, 0.0);
  std::vector<char> passive(n, 0);
  std::vector<double> res = b, w(n), z;
  double anorm = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += fabs(A[(size_t)j * m + i]);
    anorm = std::max(anorm, s);
  }
  const double tol = 10.0 * std::max(m, n) * 2.220446049250313e-16 * anorm;
  for (int outer = 0; outer < 3 * n; ++outer) {
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += A[(size_t)j * m + i] * res[i];
      w[j] = s;
    }
    int t = -1;
    double wmax = tol;
    for (int j = 0; j < n; ++j)
      if (!passive[j] && w[j] > wmax) {
        wmax = w[j];
        t = j;
      }
    if (t < 0) break;
    passive[t] = 1;
    for (int inner = 0; inner < 3 * n; ++inner) {
      std::vector<int> cols;
      for (int j = 0; j < n; ++j)
        if (passive[j]) cols.push_back(j);
      ls_subset(A, m, cols, b, z);
      bool feasible = true;
      for (double v : z) feasible = feasible && v > 0.0;
      if (feasible) {
        for (size_t c = 0; c < cols.size(); ++c) x[cols[c]] = z[c];
        break;
      }
      // step from x towards z as far as feasibility allows, then drop the columns at zero
      double step = 1.0;
      for (size_t c = 0; c < cols.size(); ++c)
        if (z[c] <= 0.0) step = std::min(step, x[cols[c]] / (x[cols[c]] - z[c]));
      for (size_t c = 0; c < cols.size(); ++c) {
        x[cols[c]] += step * (z[c] - x[cols[c]]);
        if (x[cols[c]] <= 1e-300) {
          x[cols[c]] = 0.0;
          passive[cols[c]] = 0;
        }
      }
    }
    for (int i = 0; i < m; ++i) {
      double s = b[i];
      for (int j = 0; j < n; ++j) s -= A[(size_t)j * m + i] * x[j];
      res[i] = s;
    }
  }
}

std::once_flag g_cse_once;
std::vector<double> g_cse_a, g_cse_s;
double g_cse_err = 0.0;

void fit_cse() {
  const int n = GLAD_N_CSE, m = 2000;
  g_cse_s.resize(n);
  for (int i = 0; i < n; ++i) g_cse_s[i] = pow(10.0, -5.0 + 9.0 * i / (n - 1));
  std::vector<double> u(m), A((size_t)m * n), b(m, 1.0), cs(n, 0.0), x;
  for (int r = 0; r < m; ++r) u[r] = pow(10.0, -4.0 + 7.0 * r / (m - 1));
  for (int j = 0; j < n; ++j) {
    for (int r = 0; r < m; ++r) {
      const double v = pow(u[r] * u[r] + g_cse_s[j] * g_cse_s[j], -1.5) / nfw_shape(u[r]);
      A[(size_t)j * m + r] = v;
      cs[j] += v * v;
    }
    cs[j] = sqrt(cs[j]);
    for (int r = 0; r < m; ++r) A[(size_t)j * m + r] /= cs[j];
  }
  nnls(A, m, n, b, x);
  g_cse_a.resize(n);
  for (int j = 0; j < n; ++j) g_cse_a[j] = x[j] / cs[j];
  // worst relative error on a finer grid of the same range
  double err = 0.0;
  for (int r = 0; r < 7777; ++r) {
    const double uu = pow(10.0, -4.0 + 7.0 * r / 7776.0);
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += g_cse_a[j] * pow(uu * uu + g_cse_s[j] * g_cse_s[j], -1.5);
    err = std::max(err, fabs(s / nfw_shape(uu) - 1.0));
  }
  g_cse_err = err;
}

}  // namespace

void cse_table(const double **a, const double **s) {
  std::call_once(g_cse_once, fit_cse);
  *a = g_cse_a.data();
  *s = g_cse_s.data();
}

extern "C" int glad_enfw_cse(int n, double *a, double *s, double *max_rel_err) {
  if (n < GLAD_N_CSE || !a || !s) return GLAD_N_CSE;
  const double *pa, *ps;
  cse_table(&pa, &ps);
  for (int i = 0; i < GLAD_N_CSE; ++i) {
    a[i] = pa[i];
    s[i] = ps[i];
  }
  if (max_rel_err) *max_rel_err = g_cse_err;
  return GLAD_N_CSE;
}
