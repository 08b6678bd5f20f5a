// chym_lanczos.cpp -- largest eigenvalue of the symmetric coupling matrix J.
//
// The pump threshold of the linearised equations is h_th = 1 - eps lambda_max(J)
// (the first instability of x = 0 when alpha = 1), so lambda_max sets both the
// coupling scale eps = eps_hat / lambda_max and the pump grid h = h_th (1 + dh).
// Lanczos with full re-orthogonalisation builds a tridiagonal T_m whose largest
// eigenvalue converges to lambda_max(J); that eigenvalue is isolated by Sturm
// bisection.  FP64 throughout; m <= min(N, 160).
#include <math.h>

#include <algorithm>
#include <vector>

namespace chym {

namespace {

// Number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm count).
int sturm_below(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int count = 0;
  double d = 1.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const double off = (i == 0) ? 0.0 : b[i - 1] * b[i - 1];
    d = (a[i] - x) - (i == 0 ? 0.0 : off / d);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++count;
  }
  return count;
}

double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const size_t m = a.size();
  double lo = INFINITY, hi = -INFINITY;
  for (size_t i = 0; i < m; ++i) {  // Gershgorin interval
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-14 * std::max(1.0, fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_below(a, b, mid) >= (int)m) hi = mid;  // every eigenvalue below mid
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace

double host_lambda_max(const double* J, int N) {
  if (N == 1) return J[0];
  const int m_max = std::min(N, 160);
  std::vector<std::vector<double>> V;
  std::vector<double> a, b;
  std::vector<double> v(N), w(N);
  // deterministic, non-degenerate start vector
  double nrm = 0.0;
  for (int i = 0; i < N; ++i) {
    v[i] = 1.0 + 0.37 * sin(1.0 + 2.3 * i);
    nrm += v[i] * v[i];
  }
  nrm = sqrt(nrm);
  for (int i = 0; i < N; ++i) v[i] /= nrm;
  for (int j = 0; j < m_max; ++j) {
    V.push_back(v);
    for (int i = 0; i < N; ++i) {
      double s = 0.0;
      const double* row = J + (size_t)i * N;
      for (int q = 0; q < N; ++q) s += row[q] * v[q];
      w[i] = s;
    }
    double alpha = 0.0;
    for (int i = 0; i < N; ++i) alpha += w[i] * v[i];
    a.push_back(alpha);
    // full re-orthogonalisation (twice) against every Lanczos vector
    for (int pass = 0; pass < 2; ++pass)
      for (const auto& u : V) {
        double c = 0.0;
        for (int i = 0; i < N; ++i) c += w[i] * u[i];
        for (int i = 0; i < N; ++i) w[i] -= c * u[i];
      }
    double beta = 0.0;
    for (int i = 0; i < N; ++i) beta += w[i] * w[i];
    beta = sqrt(beta);
    if (j + 1 == m_max || beta < 1e-12) break;
    b.push_back(beta);
    for (int i = 0; i < N; ++i) v[i] = w[i] / beta;
  }
  b.resize(a.size() > 0 ? a.size() - 1 : 0);
  return tridiag_max_eig(a, b);
}

}  // namespace chym
