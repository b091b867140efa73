/*
 * orc_exact.c — exact solutions, error norms and conserved quantities for the FP64 oracle.
 * TEST INFRASTRUCTURE ONLY (see dg_oracle.h).
 *
 *   - Burgers (Example 3.1): u(x,t) = u0(xi) with x = xi + t u0(xi), solved on the monotone
 *     branch by bisection (valid before the shock forms);
 *   - 1D Riemann problem of the Euler equations: the exact solver of the textbook method the paper
 *     cites for the HLLC flux (Toro): Newton on the pressure function, then sampling at x/t;
 *   - the isentropic vortex of Example 3.4(a), translated with the free stream (1, 0);
 *   - conserved quantities (mass per variable) and the discrete L2 energy of the modal state.
 */
#include "dg_oracle.h"
#include <math.h>
#include <string.h>

/* Burgers with u0(x) = a + b sin(w x + phi), period L; pre-shock solution by bisection on
 * g(xi) = xi + t u0(xi) - x, which is increasing in xi while 1 + t u0'(xi) > 0. */
double orc_burgers_exact(double x, double t, double a, double b, double w, double phi, double L) {
  (void)L;
  double umax = a + fabs(b), umin = a - fabs(b);
  double lo = x - t * umax - 1e-12, hi = x - t * umin + 1e-12;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double g = mid + t * (a + b * sin(w * mid + phi)) - x;
    if (g > 0) hi = mid; else lo = mid;
    if (hi - lo < 1e-16 * (1.0 + fabs(x))) break;
  }
  double xi = 0.5 * (lo + hi);
  return a + b * sin(w * xi + phi);
}

/* ---- exact Riemann solver (W = (rho, u, p)) ---- */
static double pfun(double g, double pstar, double rk, double pk, double ck, double* dfd) {
  if (pstar <= pk) {                                   /* rarefaction */
    double pr = pstar / pk;
    double f = 2.0 * ck / (g - 1.0) * (pow(pr, (g - 1.0) / (2.0 * g)) - 1.0);
    *dfd = 1.0 / (rk * ck) * pow(pr, -(g + 1.0) / (2.0 * g));
    return f;
  }
  double A = 2.0 / ((g + 1.0) * rk), B = (g - 1.0) / (g + 1.0) * pk;   /* shock */
  double q = sqrt(A / (pstar + B));
  *dfd = q * (1.0 - 0.5 * (pstar - pk) / (B + pstar));
  return (pstar - pk) * q;
}

int orc_riemann_exact(double g, const double* WL, const double* WR, double xi, double* W) {
  double rL = WL[0], uL = WL[1], pL = WL[2], rR = WR[0], uR = WR[1], pR = WR[2];
  double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
  if (2.0 * (cL + cR) / (g - 1.0) <= uR - uL) return -1;        /* vacuum generated */
  /* initial guess: two-rarefaction approximation */
  double z = (g - 1.0) / (2.0 * g);
  double ps = pow((cL + cR - 0.5 * (g - 1.0) * (uR - uL)) / (cL / pow(pL, z) + cR / pow(pR, z)), 1.0 / z);
  if (!(ps > 1e-14)) ps = 1e-14;
  for (int it = 0; it < 200; ++it) {
    double dL, dR;
    double f = pfun(g, ps, rL, pL, cL, &dL) + pfun(g, ps, rR, pR, cR, &dR) + (uR - uL);
    double pn = ps - f / (dL + dR);
    if (pn < 1e-14) pn = 1e-14;
    double ch = fabs(pn - ps) / (0.5 * (pn + ps));
    ps = pn;
    if (ch < 1e-15) break;
  }
  double dL, dR;
  double us = 0.5 * (uL + uR) + 0.5 * (pfun(g, ps, rR, pR, cR, &dR) - pfun(g, ps, rL, pL, cL, &dL));
  double G6 = (g - 1.0) / (g + 1.0);
  if (xi <= us) {                                               /* left of the contact */
    if (ps > pL) {
      double SL = uL - cL * sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g));
      if (xi <= SL) { W[0] = rL; W[1] = uL; W[2] = pL; }
      else { W[0] = rL * (ps / pL + G6) / (G6 * ps / pL + 1.0); W[1] = us; W[2] = ps; }
    } else {
      double SHL = uL - cL, csL = cL * pow(ps / pL, (g - 1.0) / (2.0 * g)), STL = us - csL;
      if (xi <= SHL) { W[0] = rL; W[1] = uL; W[2] = pL; }
      else if (xi >= STL) { W[0] = rL * pow(ps / pL, 1.0 / g); W[1] = us; W[2] = ps; }
      else {
        double u = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + xi);
        double cc = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - xi));
        W[0] = rL * pow(cc / cL, 2.0 / (g - 1.0));
        W[1] = u;
        W[2] = pL * pow(cc / cL, 2.0 * g / (g - 1.0));
      }
    }
  } else {                                                      /* right of the contact */
    if (ps > pR) {
      double SR = uR + cR * sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g));
      if (xi >= SR) { W[0] = rR; W[1] = uR; W[2] = pR; }
      else { W[0] = rR * (ps / pR + G6) / (G6 * ps / pR + 1.0); W[1] = us; W[2] = ps; }
    } else {
      double SHR = uR + cR, csR = cR * pow(ps / pR, (g - 1.0) / (2.0 * g)), STR = us + csR;
      if (xi >= SHR) { W[0] = rR; W[1] = uR; W[2] = pR; }
      else if (xi <= STR) { W[0] = rR * pow(ps / pR, 1.0 / g); W[1] = us; W[2] = ps; }
      else {
        double u = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + xi);
        double cc = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - xi));
        W[0] = rR * pow(cc / cR, 2.0 / (g - 1.0));
        W[1] = u;
        W[2] = pR * pow(cc / cR, 2.0 * g / (g - 1.0));
      }
    }
  }
  return 0;
}

/* Isentropic vortex of Example 3.4(a) advected by the free stream (1,0): primitive (rho,u,v,p) at
 * (x,y,t); the centre starts at (x0,y0) and the nearest periodic image is used. */
void orc_vortex_exact(double g, double x0, double y0, double beta, double Lx, double Ly, double xlo,
                      double ylo, double x, double y, double t, double* W) {
  (void)xlo; (void)ylo;
  double dx = x - t - x0, dy = y - y0;
  dx -= Lx * floor(dx / Lx + 0.5);
  dy -= Ly * floor(dy / Ly + 0.5);
  double r2 = dx * dx + dy * dy;
  double e = exp(1.0 - r2);
  double rho = pow(1.0 - (g - 1.0) / (16.0 * g * M_PI * M_PI) * beta * beta * e * e, 1.0 / (g - 1.0));
  W[0] = rho;
  W[1] = 1.0 - beta * e * dy / (2.0 * M_PI);
  W[2] = beta * e * dx / (2.0 * M_PI);
  W[3] = pow(rho, g);
}

void orc_mass(const orc_problem* p, const double* u, double* mass) {
  int nv = orc_nvars(p), nm = orc_nmodes(p);
  long ncell = (long)p->nx * (p->dim == 2 ? p->ny : 1);
  double hx = (p->x1 - p->x0) / p->nx, hy = p->dim == 2 ? (p->y1 - p->y0) / p->ny : 1.0;
  for (int v = 0; v < nv; ++v) {
    double s = 0.0;
    for (long c = 0; c < ncell; ++c) s += u[((long)v * nm) * ncell + c];
    mass[v] = s * hx * hy;                      /* int u = h * average (x hy in 2D) */
  }
}

/* sum over variables of ||u_h||^2 = sum_cells sum_modes |u^m|^2 (cell measure) * ||P_p||^2 ||P_q||^2 / 4^dim */
double orc_energy(const orc_problem* p, const double* u) {
  int nv = orc_nvars(p), nm = orc_nmodes(p);
  long ncell = (long)p->nx * (p->dim == 2 ? p->ny : 1);
  double hx = (p->x1 - p->x0) / p->nx, hy = p->dim == 2 ? (p->y1 - p->y0) / p->ny : 1.0;
  double s = 0.0;
  for (int v = 0; v < nv; ++v)
    for (int m = 0; m < nm; ++m) {
      int pp, qq;
      orc_mode_pq(p, m, &pp, &qq);
      double w = 0.5 * hx * orc_legendre_norm(pp) * (p->dim == 2 ? 0.5 * hy * orc_legendre_norm(qq) : 1.0);
      for (long c = 0; c < ncell; ++c) {
        double a = u[((long)v * nm + m) * ncell + c];
        s += w * a * a;
      }
    }
  return s;
}

/* Exact-solution kinds for orc_errors:
 *   0 Burgers sine (a, b, w, phi, L), 1 linear advection of a + b sin(w x + phi) (a, b, w, phi),
 *   2 Riemann 1D (rhoL,uL,pL, rhoR,uR,pR, xs) primitive -> conservative variable `var`,
 *   3 entropy wave (r0, A, w, u0, p0), 4 vortex (x0, y0, beta). */
static int exact_value(const orc_problem* p, int kind, const double* prm, int nprm, double t,
                       double x, double y, int var, double* out) {
  double g = p->gamma;
  if (kind == 0) {
    if (nprm < 5) return -1;
    *out = orc_burgers_exact(x, t, prm[0], prm[1], prm[2], prm[3], prm[4]);
    return 0;
  }
  if (kind == 1) {
    if (nprm < 4) return -1;
    double xx = p->dim == 2 ? (x - p->adv[0] * t) + (y - p->adv[1] * t) : x - p->adv[0] * t;
    *out = prm[0] + prm[1] * sin(prm[2] * xx + prm[3]);
    return 0;
  }
  double W[4], Uc[4];
  if (kind == 2) {
    if (nprm < 7) return -1;
    if (t <= 0) memcpy(W, x < prm[6] ? prm : prm + 3, 3 * sizeof(double));
    else if (orc_riemann_exact(g, prm, prm + 3, (x - prm[6]) / t, W)) return -1;
  } else if (kind == 3) {
    if (nprm < 5) return -1;
    W[0] = prm[0] + prm[1] * sin(prm[2] * (x - prm[3] * t));
    W[1] = prm[3];
    W[2] = prm[4];
  } else if (kind == 4) {
    if (nprm < 3) return -1;
    orc_vortex_exact(g, prm[0], prm[1], prm[2], p->x1 - p->x0, p->y1 - p->y0, p->x0, p->y0, x, y, t, W);
  } else {
    return -1;
  }
  if (p->dim == 1) {
    Uc[0] = W[0]; Uc[1] = W[0] * W[1]; Uc[2] = W[2] / (g - 1.0) + 0.5 * W[0] * W[1] * W[1];
  } else {
    Uc[0] = W[0]; Uc[1] = W[0] * W[1]; Uc[2] = W[0] * W[2];
    Uc[3] = W[3] / (g - 1.0) + 0.5 * W[0] * (W[1] * W[1] + W[2] * W[2]);
  }
  *out = Uc[var];
  return 0;
}

/* L1 = int |e|, L2 = (int e^2)^{1/2}, Linf = max over Gauss points, nq_err points per direction. */
int orc_errors(const orc_problem* p, const double* u, int kind, const double* prm, int nprm,
               double t, int nq_err, int var, double* l1, double* l2, double* linf) {
  double xq[ORC_MAXQ], wq[ORC_MAXQ];
  int nq = nq_err > 0 ? nq_err : p->k + 3;
  if (orc_gauss(nq, xq, wq)) return -1;
  int nv = orc_nvars(p), nm = orc_nmodes(p);
  long ncell = (long)p->nx * (p->dim == 2 ? p->ny : 1);
  double hx = (p->x1 - p->x0) / p->nx, hy = p->dim == 2 ? (p->y1 - p->y0) / p->ny : 1.0;
  double s1 = 0.0, s2 = 0.0, mx = 0.0;
  (void)nv;
  for (long c = 0; c < ncell; ++c) {
    int i = (int)(c % p->nx), j = (int)(c / p->nx);
    double xc = p->x0 + (i + 0.5) * hx, yc = p->dim == 2 ? p->y0 + (j + 0.5) * hy : 0.0;
    int nb = p->dim == 2 ? nq : 1;
    for (int a = 0; a < nq; ++a)
      for (int b = 0; b < nb; ++b) {
        double xi = xq[a], eta = p->dim == 2 ? xq[b] : 0.0;
        double val = 0.0;
        for (int m = 0; m < nm; ++m) {
          int pp, qq;
          orc_mode_pq(p, m, &pp, &qq);
          double phi = orc_legendre(pp, xi) * (p->dim == 2 ? orc_legendre(qq, eta) : 1.0);
          val += u[((long)var * nm + m) * ncell + c] * phi;
        }
        double ex;
        if (exact_value(p, kind, prm, nprm, t, xc + 0.5 * hx * xi, yc + 0.5 * hy * eta, var, &ex)) return -1;
        double e = fabs(val - ex);
        double w = wq[a] * 0.5 * hx * (p->dim == 2 ? wq[b] * 0.5 * hy : 1.0);
        s1 += w * e;
        s2 += w * e * e;
        if (e > mx) mx = e;
      }
  }
  *l1 = s1;
  *l2 = sqrt(s2);
  *linf = mx;
  return 0;
}
