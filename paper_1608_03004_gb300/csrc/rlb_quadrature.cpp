// Host-side quadrature of the CUDA library (section "Discretization of the momentum space using
// quadrature rules"): generalised Gauss-Laguerre (weight pbar e^-pbar, i.e. alpha = 1) for the momentum
// magnitude and Gauss-Legendre for the direction cosine.
//
// Method (Golub-Welsch setting, own implementation): the nodes are the eigenvalues of the symmetric
// tridiagonal Jacobi matrix of the orthogonal polynomials, located one by one with Sturm-sequence
// bisection in long double, then polished by Newton steps on the three-term recurrence. Weights use the
// derivative forms w = 2 / ((1 - x^2) P_n'(x)^2) (Legendre) and w = (n + 1) / (x L_n'(x)^2) (Laguerre,
// alpha = 1), which equal the paper's printed forms at the nodes.
#include <cmath>
#include <vector>

#include "rlb_internal.h"

namespace rlbq {

// Number of eigenvalues of the tridiagonal matrix (diag a, off-diagonal b[k] between k-1 and k) below lam.
static int sturm_count(const std::vector<long double>& a, const std::vector<long double>& b, long double lam) {
  int n = (int)a.size(), cnt = 0;
  long double q = a[0] - lam;
  if (q < 0) ++cnt;
  for (int k = 1; k < n; ++k) {
    if (q == 0) q = 1e-300L;
    q = (a[k] - lam) - b[k] * b[k] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

static void tridiag_eigs(const std::vector<long double>& a, const std::vector<long double>& b, long double lo,
                         long double hi, std::vector<long double>& out) {
  int n = (int)a.size();
  out.assign(n, 0.0L);
  for (int m = 0; m < n; ++m) {  // m-th smallest eigenvalue: count(<lam) goes from <= m to > m
    long double l = lo, h = hi;
    for (int it = 0; it < 200; ++it) {
      long double mid = 0.5L * (l + h);
      if (mid == l || mid == h) break;
      if (sturm_count(a, b, mid) > m)
        h = mid;
      else
        l = mid;
    }
    out[m] = 0.5L * (l + h);
  }
}

// P_n and P_{n-1} by the Bonnet recurrence.
static void legendre_pair(int n, long double x, long double& pn, long double& pn1) {
  long double p0 = 1.0L, p1 = x;
  if (n == 0) {
    pn = 1.0L;
    pn1 = 0.0L;
    return;
  }
  for (int k = 1; k < n; ++k) {
    long double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  pn = p1;
  pn1 = p0;
}

// L^(1)_n and L^(1)_{n-1}.
static void laguerre1_pair(int n, long double x, long double& ln, long double& ln1) {
  long double l0 = 1.0L, l1 = 2.0L - x;
  if (n == 0) {
    ln = 1.0L;
    ln1 = 0.0L;
    return;
  }
  for (int k = 1; k < n; ++k) {
    long double l2 = ((2 * k + 2 - x) * l1 - (k + 1) * l0) / (k + 1);
    l0 = l1;
    l1 = l2;
  }
  ln = l1;
  ln1 = l0;
}

bool gauss_legendre(int n, double* x, double* w) {
  if (n < 1) return false;
  std::vector<long double> a(n, 0.0L), b(n, 0.0L), ev;
  for (int k = 1; k < n; ++k) b[k] = k / sqrtl(4.0L * k * k - 1.0L);
  tridiag_eigs(a, b, -1.0L, 1.0L, ev);
  for (int m = 0; m < n; ++m) {
    long double z = ev[m], pn, pn1;
    for (int it = 0; it < 3; ++it) {
      legendre_pair(n, z, pn, pn1);
      long double dp = n * (pn1 - z * pn) / (1.0L - z * z);
      if (dp == 0) break;
      z -= pn / dp;
    }
    ev[m] = z;
  }
  // exact mirror symmetry of the rule
  for (int m = 0; m < n / 2; ++m) {
    long double s = 0.5L * (ev[n - 1 - m] - ev[m]);
    ev[m] = -s;
    ev[n - 1 - m] = s;
  }
  if (n % 2 == 1) ev[n / 2] = 0.0L;
  for (int m = 0; m < n; ++m) {
    long double z = ev[m], pn, pn1;
    legendre_pair(n, z, pn, pn1);
    long double dp = n * (pn1 - z * pn) / (1.0L - z * z);
    x[m] = (double)z;
    w[m] = (double)(2.0L / ((1.0L - z * z) * dp * dp));
    if (m > 0 && !(x[m] > x[m - 1])) return false;
  }
  return true;
}

bool gauss_laguerre1(int n, double* x, double* w) {
  if (n < 1) return false;
  std::vector<long double> a(n), b(n, 0.0L), ev;
  for (int k = 0; k < n; ++k) a[k] = 2.0L * k + 2.0L;
  for (int k = 1; k < n; ++k) b[k] = sqrtl((long double)k * (k + 1));
  tridiag_eigs(a, b, 0.0L, 4.0L * n + 4.0L, ev);
  for (int m = 0; m < n; ++m) {
    long double z = ev[m], ln, ln1;
    for (int it = 0; it < 3; ++it) {
      laguerre1_pair(n, z, ln, ln1);
      long double dl = (n * ln - (n + 1) * ln1) / z;
      if (dl == 0) break;
      z -= ln / dl;
    }
    laguerre1_pair(n, z, ln, ln1);
    long double dl = (n * ln - (n + 1) * ln1) / z;
    x[m] = (double)z;
    w[m] = (double)((n + 1) / (z * dl * dl));
    if (m > 0 && !(x[m] > x[m - 1])) return false;
  }
  return true;
}

double laguerre1(int l, double x) {
  long double ln, ln1;
  laguerre1_pair(l, x, ln, ln1);
  return (double)ln;
}

double legendre(int k, double x) {
  long double pn, pn1;
  legendre_pair(k, x, pn, pn1);
  return (double)pn;
}

}  // namespace rlbq
