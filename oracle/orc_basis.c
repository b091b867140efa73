/*
 * orc_basis.c — Legendre polynomials and Gauss–Legendre rules for the FP64 oracle.
 * TEST INFRASTRUCTURE ONLY (see dg_oracle.h).
 *
 * The modal basis of Eq. (GLbasisequation) is the Legendre family P_l on the reference cell [-1,1],
 * P_l(1) = 1. Values use Bonnet's three-term recurrence; derivatives of any order use the exact
 * monomial coefficients of P_l (small dyadic rationals for l <= 8, so the coefficients are exact in
 * FP64) differentiated term by term. Gauss nodes come from Newton's method on P_n.
 */
#include "dg_oracle.h"
#include <math.h>
#include <string.h>

#define MONO_MAX 10

/* Monomial coefficients c[n][i] of P_n(x) = sum_i c[n][i] x^i, from
 * (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}. */
static void legendre_monomials(double c[MONO_MAX + 1][MONO_MAX + 1]) {
  memset(c, 0, sizeof(double) * (MONO_MAX + 1) * (MONO_MAX + 1));
  c[0][0] = 1.0;
  c[1][1] = 1.0;
  for (int n = 1; n < MONO_MAX; ++n)
    for (int i = 0; i <= n + 1; ++i) {
      double a = (i >= 1) ? (2.0 * n + 1.0) * c[n][i - 1] : 0.0;
      double b = (double)n * c[n - 1][i];
      c[n + 1][i] = (a - b) / (double)(n + 1);
    }
}

double orc_legendre(int n, double x) {
  if (n == 0) return 1.0;
  double pm = 1.0, p = x;
  for (int j = 1; j < n; ++j) {
    double pn = ((2.0 * j + 1.0) * x * p - (double)j * pm) / (double)(j + 1);
    pm = p;
    p = pn;
  }
  return p;
}

/* d^m/dx^m P_n(x): differentiate the monomial expansion m times, evaluate by Horner. */
double orc_legendre_deriv(int n, int m, double x) {
  if (n > MONO_MAX || n < 0 || m < 0) return NAN;
  if (m > n) return 0.0;
  double c[MONO_MAX + 1][MONO_MAX + 1];
  legendre_monomials(c);
  double d[MONO_MAX + 1];
  for (int i = 0; i <= n; ++i) d[i] = c[n][i];
  int deg = n;
  for (int r = 0; r < m; ++r) {
    for (int i = 0; i < deg; ++i) d[i] = d[i + 1] * (double)(i + 1);
    d[deg] = 0.0;
    --deg;
  }
  double s = 0.0;
  for (int i = deg; i >= 0; --i) s = s * x + d[i];
  return s;
}

/* Gauss–Legendre nodes (ascending) and weights for n points: Newton iteration on P_n from the
 * Chebyshev-like guess cos(pi (i - 1/4)/(n + 1/2)); P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1);
 * weights w = 2 / ((1 - x^2) P_n'(x)^2). */
int orc_gauss(int n, double* x, double* w) {
  if (n < 1 || n > ORC_MAXQ) return -1;
  if (n == 1) { x[0] = 0.0; w[0] = 2.0; return 0; }
  for (int i = 1; i <= n; ++i) {
    double z = cos(M_PI * (i - 0.25) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double pn = orc_legendre(n, z), pm = orc_legendre(n - 1, z);
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    double pn = orc_legendre(n, z), pm = orc_legendre(n - 1, z);
    dp = n * (z * pn - pm) / (z * z - 1.0);
    x[n - i] = z;                              /* cos decreases with i: store ascending */
    w[n - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return 0;
}

/* int_{-1}^{1} P_n(x)^2 dx by an (n+2)-point Gauss rule (exact for degree 2n). */
double orc_legendre_norm(int n) {
  double x[ORC_MAXQ], w[ORC_MAXQ];
  int q = n + 2;
  if (q > ORC_MAXQ) q = ORC_MAXQ;
  orc_gauss(q, x, w);
  double s = 0.0;
  for (int i = 0; i < q; ++i) {
    double v = orc_legendre(n, x[i]);
    s += w[i] * v * v;
  }
  return s;
}
