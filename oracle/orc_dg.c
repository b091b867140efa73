/*
 * orc_dg.c — DG spatial operator, jump filter, SSP-RK3 stepping, CFL and L2 projection for the FP64
 * oracle. TEST INFRASTRUCTURE ONLY (see dg_oracle.h).
 *
 * Everything is written as plain loops over cells in the paper's order: the DG residual of
 * Eq. (scheme:DG) (1D) and of the 2D weak form (Section 2.2, with the local viscosity term dropped:
 * it enters only through the filter), then the Shu–Osher combination of Eq. (rkdg1)/(err_rk1), then
 * the jump filter of Eqs. (para:damp2)-(para:damp21)/(timespli:1dscalar) (1D) or
 * (para:2ddamp), (para:damp22d)-(para:damp22d1) (2D), systems by Eqs. (para:dampsystems1d)-(timespli:sys),
 * in the literal form with c_f^l and the (2/h)^2 l(l+1) or (2/hx)(2/hy) lambda_{p,q} factors.
 * Face fluxes are recomputed by both neighbours with the same argument order, so they agree bitwise.
 */
#include "dg_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int nv, nm, nq, k;
  int mp[ORC_MAXNM], mq[ORC_MAXNM];            /* (p,q) degrees of mode m */
  double xq[ORC_MAXQ], wq[ORC_MAXQ];            /* Gauss rule on [-1,1] */
  double P[ORC_MAXK + 1][ORC_MAXQ];             /* P_l(x_q) */
  double dP[ORC_MAXK + 1][ORC_MAXQ];            /* P_l'(x_q) */
  double Pe[2][ORC_MAXK + 1];                   /* P_l(-1), P_l(+1) */
  double De[2][ORC_MAXK + 1][ORC_MAXK + 1];     /* [side][l][r] = d^r P_l at -1 (side 0) / +1 (side 1) */
  double nrm[ORC_MAXK + 1];                     /* int P_l^2 */
  double hx, hy;
  long ncell;
} ctx_t;

static int g_threads = 1;
void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_threads; }

int orc_nmodes(const orc_problem* p) {
  if (p->dim == 1) return p->k + 1;
  if (p->basis == ORC_BASIS_P) return (p->k + 1) * (p->k + 2) / 2;
  return (p->k + 1) * (p->k + 1);
}

void orc_mode_pq(const orc_problem* p, int m, int* pdeg, int* qdeg) {
  if (p->dim == 1) { *pdeg = m; *qdeg = 0; return; }
  int idx = 0;
  for (int q = 0; q <= p->k; ++q)
    for (int pp = 0; pp <= p->k; ++pp) {
      if (p->basis == ORC_BASIS_P && pp + q > p->k) continue;
      if (idx == m) { *pdeg = pp; *qdeg = q; return; }
      ++idx;
    }
  *pdeg = -1; *qdeg = -1;
}

long orc_state_size(const orc_problem* p) {
  return (long)orc_nvars(p) * orc_nmodes(p) * (long)p->nx * (p->dim == 2 ? p->ny : 1);
}

static double fact(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

static void make_ctx(const orc_problem* p, ctx_t* c) {
  memset(c, 0, sizeof(*c));
  c->k = p->k;
  c->nv = orc_nvars(p);
  c->nm = orc_nmodes(p);
  c->nq = p->nq > 0 ? p->nq : p->k + 1;
  for (int m = 0; m < c->nm; ++m) orc_mode_pq(p, m, &c->mp[m], &c->mq[m]);
  orc_gauss(c->nq, c->xq, c->wq);
  for (int l = 0; l <= p->k; ++l) {
    for (int q = 0; q < c->nq; ++q) {
      c->P[l][q] = orc_legendre(l, c->xq[q]);
      c->dP[l][q] = orc_legendre_deriv(l, 1, c->xq[q]);
    }
    c->Pe[0][l] = orc_legendre(l, -1.0);
    c->Pe[1][l] = orc_legendre(l, 1.0);
    for (int r = 0; r <= p->k; ++r) {
      c->De[0][l][r] = orc_legendre_deriv(l, r, -1.0);
      c->De[1][l][r] = orc_legendre_deriv(l, r, 1.0);
    }
    c->nrm[l] = orc_legendre_norm(l);
  }
  c->hx = (p->x1 - p->x0) / p->nx;
  c->hy = p->dim == 2 ? (p->y1 - p->y0) / p->ny : 1.0;
  c->ncell = (long)p->nx * (p->dim == 2 ? p->ny : 1);
}

#define U(u, v, m, cell) (u)[((long)(v) * c->nm + (m)) * c->ncell + (cell)]

/* Neighbour cell across a face: dir 0 = x, 1 = y; side 0 = low, 1 = high. -1 = outflow boundary. */
static long neighbour(const orc_problem* p, int i, int j, int dir, int side) {
  int nx = p->nx, ny = p->dim == 2 ? p->ny : 1;
  if (dir == 0) {
    int ii = side ? i + 1 : i - 1;
    if (ii < 0 || ii >= nx) {
      if (p->bc[side] == ORC_BC_OUTFLOW) return -1;
      ii = (ii + nx) % nx;
    }
    return (long)ii + (long)nx * j;
  }
  int jj = side ? j + 1 : j - 1;
  if (jj < 0 || jj >= ny) {
    if (p->bc[2 + side] == ORC_BC_OUTFLOW) return -1;
    jj = (jj + ny) % ny;
  }
  return (long)i + (long)nx * jj;
}

/* Value of every variable of the cell polynomial at reference point (xi, eta). */
static void eval_cell(const orc_problem* p, const ctx_t* c, const double* u, long cell, double xi,
                      double eta, double* val) {
  for (int v = 0; v < c->nv; ++v) {
    double s = 0.0;
    for (int m = 0; m < c->nm; ++m) {
      double b = orc_legendre(c->mp[m], xi);
      if (p->dim == 2) b *= orc_legendre(c->mq[m], eta);
      s += U(u, v, m, cell) * b;
    }
    val[v] = s;
  }
}

/* The outflow ghost cell: the constant state equal to the interior cell's average. */
static void cell_average(const ctx_t* c, const double* u, long cell, double* val) {
  for (int v = 0; v < c->nv; ++v) val[v] = U(u, v, 0, cell);
}

void orc_eval(const orc_problem* p, const double* u, int cell, double xi, double eta, double* val) {
  ctx_t c;
  make_ctx(p, &c);
  eval_cell(p, &c, u, cell, xi, eta, val);
}

/* Local Lax–Friedrichs flux (Section 3): 1/2 (f(uL)+f(uR)) - 1/2 alpha (uR - uL),
 * alpha = max of the two spectral radii. */
static void llf(const orc_problem* p, int dir, const double* uL, const double* uR, double* fh) {
  double fL[ORC_MAXNV], fR[ORC_MAXNV];
  orc_flux(p, dir, uL, fL);
  orc_flux(p, dir, uR, fR);
  double aL = orc_wave_speed(p, dir, uL), aR = orc_wave_speed(p, dir, uR);
  double a = aL > aR ? aL : aR;
  if (isnan(aL) || isnan(aR)) a = NAN;
  int nv = orc_nvars(p);
  for (int v = 0; v < nv; ++v) fh[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * a * (uR[v] - uL[v]);
}

/* ------------------------------------------------------------------------------------------ */
/* DG residual R = M^{-1} [ (f(u_h), v_x)_K - <f^, v>_{dK} ]  (Eq. scheme:DG), per mode.       */
/* ------------------------------------------------------------------------------------------ */
static void residual_1d(const orc_problem* p, const ctx_t* c, const double* u, double* R) {
  const double h = c->hx;
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (long i = 0; i < c->ncell; ++i) {
    double vol[ORC_MAXNV][ORC_MAXK + 1];
    memset(vol, 0, sizeof(vol));
    /* volume term: (f(u_h), d/dx P_l)_K = int_{-1}^{1} f(u_h(xi)) P_l'(xi) dxi */
    for (int q = 0; q < c->nq; ++q) {
      double uq[ORC_MAXNV], fq[ORC_MAXNV];
      eval_cell(p, c, u, i, c->xq[q], 0.0, uq);
      orc_flux(p, 0, uq, fq);
      for (int v = 0; v < c->nv; ++v)
        for (int l = 0; l <= c->k; ++l) vol[v][l] += c->wq[q] * fq[v] * c->dP[l][q];
    }
    /* faces j+1/2 and j-1/2 */
    double own_r[ORC_MAXNV], own_l[ORC_MAXNV], nb[ORC_MAXNV], fr[ORC_MAXNV], fl[ORC_MAXNV];
    eval_cell(p, c, u, i, 1.0, 0.0, own_r);
    eval_cell(p, c, u, i, -1.0, 0.0, own_l);
    long ir = neighbour(p, (int)i, 0, 0, 1), il = neighbour(p, (int)i, 0, 0, 0);
    /* outflow: the ghost cell holds the constant state equal to this cell's average */
    if (ir >= 0) eval_cell(p, c, u, ir, -1.0, 0.0, nb); else cell_average(c, u, i, nb);
    llf(p, 0, own_r, nb, fr);
    if (il >= 0) eval_cell(p, c, u, il, 1.0, 0.0, nb); else cell_average(c, u, i, nb);
    llf(p, 0, nb, own_l, fl);
    for (int v = 0; v < c->nv; ++v)
      for (int l = 0; l <= c->k; ++l) {
        double rhs = vol[v][l] - fr[v] * c->Pe[1][l] + fl[v] * c->Pe[0][l];
        double mass = 0.5 * h * c->nrm[l];               /* (P_l, P_l)_{K_j} */
        U(R, v, l, i) = rhs / mass;
      }
  }
}

static void residual_2d(const orc_problem* p, const ctx_t* c, const double* u, double* R) {
  const double hx = c->hx, hy = c->hy;
  const int nx = p->nx;
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (long cell = 0; cell < c->ncell; ++cell) {
    int i = (int)(cell % nx), j = (int)(cell / nx);
    double acc[ORC_MAXNV][ORC_MAXNM];
    memset(acc, 0, sizeof(acc));
    /* volume term: (F(u_h), grad phi)_K with phi = P_p(xi) P_q(eta), dx dy = hx hy/4 dxi deta */
    for (int a = 0; a < c->nq; ++a)
      for (int b = 0; b < c->nq; ++b) {
        double uq[ORC_MAXNV], fx[ORC_MAXNV], fy[ORC_MAXNV];
        eval_cell(p, c, u, cell, c->xq[a], c->xq[b], uq);
        orc_flux(p, 0, uq, fx);
        orc_flux(p, 1, uq, fy);
        double wgt = 0.25 * hx * hy * c->wq[a] * c->wq[b];
        for (int m = 0; m < c->nm; ++m) {
          int pp = c->mp[m], qq = c->mq[m];
          double phix = (2.0 / hx) * c->dP[pp][a] * c->P[qq][b];
          double phiy = c->P[pp][a] * (2.0 / hy) * c->dP[qq][b];
          for (int v = 0; v < c->nv; ++v) acc[v][m] += wgt * (fx[v] * phix + fy[v] * phiy);
        }
      }
    /* boundary term: - int_{dK} F^ . n phi ds, each edge by the same Gauss rule, ds = h/2 dt */
    long nb_r = neighbour(p, i, j, 0, 1), nb_l = neighbour(p, i, j, 0, 0);
    long nb_t = neighbour(p, i, j, 1, 1), nb_b = neighbour(p, i, j, 1, 0);
    for (int g = 0; g < c->nq; ++g) {
      double s = c->xq[g];
      double in[ORC_MAXNV], out[ORC_MAXNV], fh[ORC_MAXNV];
      /* right edge, n = (+1, 0): left state = this cell at xi=+1, right state = neighbour at xi=-1 */
      eval_cell(p, c, u, cell, 1.0, s, in);
      if (nb_r >= 0) eval_cell(p, c, u, nb_r, -1.0, s, out); else cell_average(c, u, cell, out);
      llf(p, 0, in, out, fh);
      for (int m = 0; m < c->nm; ++m) {
        double phi = c->Pe[1][c->mp[m]] * c->P[c->mq[m]][g];
        for (int v = 0; v < c->nv; ++v) acc[v][m] -= 0.5 * hy * c->wq[g] * fh[v] * phi;
      }
      /* left edge, n = (-1, 0): left state = neighbour at xi=+1, right state = this cell at xi=-1 */
      eval_cell(p, c, u, cell, -1.0, s, in);
      if (nb_l >= 0) eval_cell(p, c, u, nb_l, 1.0, s, out); else cell_average(c, u, cell, out);
      llf(p, 0, out, in, fh);
      for (int m = 0; m < c->nm; ++m) {
        double phi = c->Pe[0][c->mp[m]] * c->P[c->mq[m]][g];
        for (int v = 0; v < c->nv; ++v) acc[v][m] += 0.5 * hy * c->wq[g] * fh[v] * phi;
      }
      /* top edge, n = (0, +1) */
      eval_cell(p, c, u, cell, s, 1.0, in);
      if (nb_t >= 0) eval_cell(p, c, u, nb_t, s, -1.0, out); else cell_average(c, u, cell, out);
      llf(p, 1, in, out, fh);
      for (int m = 0; m < c->nm; ++m) {
        double phi = c->P[c->mp[m]][g] * c->Pe[1][c->mq[m]];
        for (int v = 0; v < c->nv; ++v) acc[v][m] -= 0.5 * hx * c->wq[g] * fh[v] * phi;
      }
      /* bottom edge, n = (0, -1) */
      eval_cell(p, c, u, cell, s, -1.0, in);
      if (nb_b >= 0) eval_cell(p, c, u, nb_b, s, 1.0, out); else cell_average(c, u, cell, out);
      llf(p, 1, out, in, fh);
      for (int m = 0; m < c->nm; ++m) {
        double phi = c->P[c->mp[m]][g] * c->Pe[0][c->mq[m]];
        for (int v = 0; v < c->nv; ++v) acc[v][m] += 0.5 * hx * c->wq[g] * fh[v] * phi;
      }
    }
    for (int m = 0; m < c->nm; ++m) {
      double mass = 0.25 * hx * hy * c->nrm[c->mp[m]] * c->nrm[c->mq[m]];
      for (int v = 0; v < c->nv; ++v) U(R, v, m, cell) = acc[v][m] / mass;
    }
  }
}

void orc_residual(const orc_problem* p, const double* u, double* R) {
  ctx_t c;
  make_ctx(p, &c);
  if (p->dim == 1) residual_1d(p, &c, u, R); else residual_2d(p, &c, u, R);
}

/* ------------------------------------------------------------------------------------------ */
/* The jump filter                                                                            */
/* ------------------------------------------------------------------------------------------ */

/* Physical derivative d^r/dx^r of variable v of a 1D cell at xi = -1 (side 0) or +1 (side 1). */
static double end_deriv_1d(const ctx_t* c, const double* u, int v, long cell, int side, int r) {
  double s = 0.0;
  for (int l = 0; l <= c->k; ++l) s += U(u, v, l, cell) * c->De[side][l][r];
  return pow(2.0 / c->hx, r) * s;
}

/* sigma^l of Eqs. (para:damp2)-(para:damp21), maximised over components (Eq. para:dampsystems1d). */
static void sigma_1d(const orc_problem* p, const ctx_t* c, const double* u, long i, const double* ninf,
                     double* sig) {
  const double h = c->hx;
  double J[ORC_MAXNV][ORC_MAXK + 1];
  long il = neighbour(p, (int)i, 0, 0, 0), ir = neighbour(p, (int)i, 0, 0, 1);
  for (int v = 0; v < c->nv; ++v)
    for (int r = 0; r <= c->k; ++r) {
      /* ||[d^r u]||_{dK_j} = |w(x_{j-1/2}^+) - w(x_{j-1/2}^-)| + |w(x_{j+1/2}^+) - w(x_{j+1/2}^-)| */
      /* outflow ghost: constant state = this cell's average (value u_bar, derivatives 0) */
      const double ghost = (r == 0) ? U(u, v, 0, i) : 0.0;
      double dl_nb = il >= 0 ? end_deriv_1d(c, u, v, il, 1, r) : ghost;
      double dr_nb = ir >= 0 ? end_deriv_1d(c, u, v, ir, 0, r) : ghost;
      double jl = fabs(end_deriv_1d(c, u, v, i, 0, r) - dl_nb);
      double jr = fabs(dr_nb - end_deriv_1d(c, u, v, i, 1, r));
      J[v][r] = jl + jr;
    }
  double ubar[ORC_MAXNV];
  for (int v = 0; v < c->nv; ++v) ubar[v] = U(u, v, 0, i);
  double beta = orc_wave_speed(p, 0, ubar);          /* |f'(u_bar)| or the spectral radius */
  double Hbar = orc_enthalpy(p, ubar);               /* Euler: 1/H_bar factor (Section 3.1) */
  sig[0] = 0.0;                                      /* sigma^0 = 0: cell averages untouched */
  for (int l = 1; l <= c->k; ++l) {
    if (p->filter_kind == ORC_FILTER_OEDG) {
      /* sigma^{l,OE} = sigma^{OE}_{j,l} / h^2, each component with its own c_f^OE */
      double best = 0.0;
      for (int v = 0; v < c->nv; ++v) {
        double cf = ninf[v] > 0.0 ? beta / (2.0 * (2 * c->k - 1) * ninf[v]) : 0.0;
        double s = h * J[v][0];
        for (int m = 1; m <= l; ++m) s += (2.0 * m + 1.0) / fact(m) * pow(h, m + 1) * J[v][m];
        s = cf * s / (h * h);
        if (s > best || isnan(s)) best = s;
      }
      sig[l] = best;
      continue;
    }
    /* the jump filter sums the jumps up to order l (Eq. para:damp21); the global coefficient of
     * Eq. (para:damp) takes every order up to k, for every mode */
    const int top = p->filter_kind == ORC_FILTER_GLOBAL ? c->k : l;
    double cf = beta / (4.0 * l * (l + 1)) / Hbar;   /* c_f^l */
    double best = 0.0;
    for (int v = 0; v < c->nv; ++v) {
      double s = h * J[v][0];
      for (int m = 1; m <= top; ++m) s += m * (m + 1) * pow(h, m + 1) * J[v][m];
      s *= cf;                                       /* sigma_{j,l}(u^(v)) */
      if (s > best || isnan(s)) best = s;
    }
    sig[l] = best * (2.0 / h) * (2.0 / h) * l * (l + 1);
  }
}

/* d^{a1}_x d^{a2}_y of variable v of a 2D cell at the corner (xi, eta) = (+-1, +-1). */
static double corner_deriv_2d(const ctx_t* c, const double* u, int v, long cell, int sx, int sy,
                              int a1, int a2) {
  double s = 0.0;
  for (int m = 0; m < c->nm; ++m) s += U(u, v, m, cell) * c->De[sx][c->mp[m]][a1] * c->De[sy][c->mq[m]][a2];
  return pow(2.0 / c->hx, a1) * pow(2.0 / c->hy, a2) * s;
}

/* sigma for every mode of a 2D cell, Eqs. (para:damp22d)-(para:damp22d1) with the Euler choice of
 * (c_fx, c_fy) of Section 3.2 (scalar laws: H_bar = 1), edge norms by the trapezoidal rule. */
static void sigma_2d(const orc_problem* p, const ctx_t* c, const double* u, long cell, const double* ninf,
                     double* sig) {
  const double hx = c->hx, hy = c->hy;
  const int k = c->k, nx = p->nx;
  int i = (int)(cell % nx), j = (int)(cell / nx);
  long nl = neighbour(p, i, j, 0, 0), nr = neighbour(p, i, j, 0, 1);
  long nb = neighbour(p, i, j, 1, 0), nt = neighbour(p, i, j, 1, 1);
  /* JV[v][a1][a2]: ||[d^alpha u]|| over the vertical edges; JH over the horizontal edges. */
  double JV[ORC_MAXNV][ORC_MAXK + 1][ORC_MAXK + 1], JH[ORC_MAXNV][ORC_MAXK + 1][ORC_MAXK + 1];
  for (int v = 0; v < c->nv; ++v)
    for (int a1 = 0; a1 <= k; ++a1)
      for (int a2 = 0; a2 <= k; ++a2) {
        double sv = 0.0, sh = 0.0;
        /* outflow ghost: constant state = this cell's average (value u_bar, derivatives 0) */
        const double ghost = (a1 == 0 && a2 == 0) ? U(u, v, 0, cell) : 0.0;
        for (int cy = 0; cy <= 1; ++cy) {        /* the two corners of each vertical edge */
          double gl = nl >= 0 ? corner_deriv_2d(c, u, v, nl, 1, cy, a1, a2) : ghost;
          double gr = nr >= 0 ? corner_deriv_2d(c, u, v, nr, 0, cy, a1, a2) : ghost;
          sv += 0.5 * fabs(corner_deriv_2d(c, u, v, cell, 0, cy, a1, a2) - gl);
          sv += 0.5 * fabs(gr - corner_deriv_2d(c, u, v, cell, 1, cy, a1, a2));
        }
        for (int cx = 0; cx <= 1; ++cx) {        /* the two corners of each horizontal edge */
          double gb = nb >= 0 ? corner_deriv_2d(c, u, v, nb, cx, 1, a1, a2) : ghost;
          double gt = nt >= 0 ? corner_deriv_2d(c, u, v, nt, cx, 0, a1, a2) : ghost;
          sh += 0.5 * fabs(corner_deriv_2d(c, u, v, cell, cx, 0, a1, a2) - gb);
          sh += 0.5 * fabs(gt - corner_deriv_2d(c, u, v, cell, cx, 1, a1, a2));
        }
        JV[v][a1][a2] = sv;
        JH[v][a1][a2] = sh;
      }
  double ubar[ORC_MAXNV];
  for (int v = 0; v < c->nv; ++v) ubar[v] = U(u, v, 0, cell);
  double bx = orc_wave_speed(p, 0, ubar), by = orc_wave_speed(p, 1, ubar);
  double Hbar = orc_enthalpy(p, ubar);
  if (p->filter_study & 3) {
    /* study readings: wave speeds over the cell's Gauss points, Hbar as the average of H */
    double hsum = 0.0, wsum = 0.0;
    for (int a = 0; a < c->nq; ++a)
      for (int b = 0; b < c->nq; ++b) {
        double val[ORC_MAXNV];
        eval_cell(p, c, u, cell, c->xq[a], c->xq[b], val);
        if (p->filter_study & 1) {
          bx = fmax(bx, orc_wave_speed(p, 0, val));
          by = fmax(by, orc_wave_speed(p, 1, val));
        }
        hsum += c->wq[a] * c->wq[b] * orc_enthalpy(p, val);
        wsum += c->wq[a] * c->wq[b];
      }
    if (p->filter_study & 1)
      for (int e = 0; e < 4; ++e)
        for (int g = 0; g < c->nq; ++g) {
          const double xi = e < 2 ? (e == 0 ? -1.0 : 1.0) : c->xq[g];
          const double eta = e < 2 ? c->xq[g] : (e == 2 ? -1.0 : 1.0);
          double val[ORC_MAXNV];
          eval_cell(p, c, u, cell, xi, eta, val);
          bx = fmax(bx, orc_wave_speed(p, 0, val));
          by = fmax(by, orc_wave_speed(p, 1, val));
        }
    if (p->filter_study & 2) Hbar = hsum / wsum;
  }
  for (int m = 0; m < c->nm; ++m) {
    int pp = c->mp[m], qq = c->mq[m], l = pp + qq;
    if (l == 0) { sig[m] = 0.0; continue; }
    if (p->filter_kind == ORC_FILTER_OEDG) {
      /* The paper states the OEDG damping in 1D only; in 2D each direction takes its edges as the
       * jump filter does: sigma = c_f^OE [beta^x (h_x J^V_0 + sum_{m=1..l} (2m+1)/m! h_x^{m+1}
       * S^V_m) / h_x^2 + beta^y (the same with H, h_y) / h_y^2] with beta / c_f^OE shared, so that
       * y-invariant data give the 1D value. */
      double best = 0.0;
      for (int v = 0; v < c->nv; ++v) {
        double cf = ninf[v] > 0.0 ? 1.0 / (2.0 * (2 * k - 1) * ninf[v]) : 0.0;
        double sx = hx * JV[v][0][0], sy = hy * JH[v][0][0];
        for (int mm = 1; mm <= l; ++mm) {
          double tv = 0.0, th = 0.0;
          for (int a1 = 0; a1 <= k; ++a1) {
            int a2 = mm - a1;
            if (a2 < 0 || a2 > k) continue;
            tv += JV[v][a1][a2];
            th += JH[v][a1][a2];
          }
          sx += (2.0 * mm + 1.0) / fact(mm) * pow(hx, mm + 1) * tv;
          sy += (2.0 * mm + 1.0) / fact(mm) * pow(hy, mm + 1) * th;
        }
        double s = cf * (bx * sx / (hx * hx) + by * sy / (hy * hy));
        if (s > best || isnan(s)) best = s;
      }
      sig[m] = best;
      continue;
    }
    /* the global coefficient of Eq. (para:damp) (2D: Eq. eq:2dalljumpvis1) takes every derivative
     * order the space holds (|alpha| up to 2k with alpha_1, alpha_2 <= k), for every mode */
    const int top = p->filter_kind == ORC_FILTER_GLOBAL ? 2 * k : l;
    double lam = pp * (pp + 1) + qq * (qq + 1);      /* lambda_{p,q} */
    double cfx = hy * bx / (4.0 * lam * Hbar);       /* c_{f,x}^{p,q} */
    double cfy = hx * by / (4.0 * lam * Hbar);       /* c_{f,y}^{p,q} */
    double best = 0.0, bestx = 0.0, besty = 0.0;
    for (int v = 0; v < c->nv; ++v) {
      double sx = hx * JV[v][0][0], sy = hy * JH[v][0][0];
      for (int mm = 1; mm <= top; ++mm) {
        double tv = 0.0, th = 0.0;
        for (int a1 = 0; a1 <= k; ++a1) {            /* |alpha| = mm */
          int a2 = mm - a1;
          if (a2 < 0 || a2 > k) continue;
          tv += JV[v][a1][a2];
          th += JH[v][a1][a2];
        }
        sx += mm * (mm + 1) * pow(hx, mm + 1) * tv;
        sy += mm * (mm + 1) * pow(hy, mm + 1) * th;
      }
      double s = cfx * sx + cfy * sy;                /* sigma_{i,j,l}(u^(v)) */
      if (p->filter_study & 4) {                     /* study: per-direction maxima, then added */
        if (cfx * sx > bestx || isnan(sx)) bestx = cfx * sx;
        if (cfy * sy > besty || isnan(sy)) besty = cfy * sy;
        best = bestx + besty;
        continue;
      }
      if (s > best || isnan(s)) best = s;
    }
    sig[m] = best * (2.0 / hx) * (2.0 / hy) * lam;
  }
}

/* ||u_v - avg(u_v)||_{L^inf(Omega)} per variable for the OEDG coefficient: avg is the domain average
 * (the mean of the cell averages on the uniform mesh), the maximum is taken at the volume Gauss
 * points of every cell (the k+1-point rule per direction). */
static void oedg_norms(const orc_problem* p, const ctx_t* c, const double* u, double* ninf) {
  for (int v = 0; v < c->nv; ++v) {
    double avg = 0.0;
    for (long cell = 0; cell < c->ncell; ++cell) avg += U(u, v, 0, cell);
    avg /= (double)c->ncell;
    double mx = 0.0;
    for (long cell = 0; cell < c->ncell; ++cell)
      for (int a = 0; a < c->nq; ++a)
        for (int b = 0; b < (p->dim == 2 ? c->nq : 1); ++b) {
          double val = 0.0;
          for (int m = 0; m < c->nm; ++m)
            val += U(u, v, m, cell) * c->P[c->mp[m]][a] * (p->dim == 2 ? c->P[c->mq[m]][b] : 1.0);
          double d = fabs(val - avg);
          if (d > mx || isnan(d)) mx = d;
        }
    ninf[v] = mx;
  }
}

void orc_oedg_norms(const orc_problem* p, const double* u, double* ninf) {
  ctx_t c;
  make_ctx(p, &c);
  oedg_norms(p, &c, u, ninf);
}

void orc_filter_sigma(const orc_problem* p, const double* u, double* sigma) {
  ctx_t c;
  make_ctx(p, &c);
  double ninf[ORC_MAXNV] = {0};
  if (p->filter_kind == ORC_FILTER_OEDG) oedg_norms(p, &c, u, ninf);
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (long cell = 0; cell < c.ncell; ++cell) {
    double s[ORC_MAXNM];
    if (p->dim == 1) sigma_1d(p, &c, u, cell, ninf, s); else sigma_2d(p, &c, u, cell, ninf, s);
    for (int m = 0; m < c.nm; ++m) sigma[(long)m * c.ncell + cell] = s[m];
  }
}

/* u^l <- exp(-sigma^l dt) u^l  (Eqs. timespli:1dscalar, timespli:sys and the 2D counterpart). */
void orc_filter(const orc_problem* p, const double* u, double dt, double* out) {
  ctx_t cc;
  make_ctx(p, &cc);
  const ctx_t* c = &cc;
  double ninf[ORC_MAXNV] = {0};
  if (p->filter_kind == ORC_FILTER_OEDG) oedg_norms(p, c, u, ninf);
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (long cell = 0; cell < c->ncell; ++cell) {
    double s[ORC_MAXNM];
    if (p->dim == 1) sigma_1d(p, c, u, cell, ninf, s); else sigma_2d(p, c, u, cell, ninf, s);
    for (int m = 0; m < c->nm; ++m) {
      double f = (m == 0) ? 1.0 : exp(-s[m] * dt);
      for (int v = 0; v < c->nv; ++v) U(out, v, m, cell) = f * U(u, v, m, cell);
    }
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Hybrid limiter of Algorithm 1 (Section 2.4): the jump indicator eta_j flags troubled cells, on  */
/* which the DG solution is blended with its jump-filtered version u^lim by the weight            */
/* omega_j = (max eta - eta_j) / (max eta - 1); elsewhere the DG solution is kept unfiltered.      */
/* The indicator is taken on the first conservative variable (density for Euler); 1D:             */
/* eta_j = (|[u]_{j-1/2}| + |[u]_{j+1/2}|) / (2 h); 2D: the same per direction with each edge's    */
/* jump averaged over its two corners, eta = J^V / (2 h_x) + J^H / (2 h_y), so that y-invariant   */
/* data give the 1D value. Outflow ghosts hold the cell average, as for the filter.              */
/* ------------------------------------------------------------------------------------------ */
static double eta_cell(const orc_problem* p, const ctx_t* c, const double* u, long cell) {
  if (p->dim == 1) {
    long il = neighbour(p, (int)cell, 0, 0, 0), ir = neighbour(p, (int)cell, 0, 0, 1);
    const double ghost = U(u, 0, 0, cell);
    double nl = il >= 0 ? end_deriv_1d(c, u, 0, il, 1, 0) : ghost;
    double nr = ir >= 0 ? end_deriv_1d(c, u, 0, ir, 0, 0) : ghost;
    double jl = fabs(end_deriv_1d(c, u, 0, cell, 0, 0) - nl);
    double jr = fabs(nr - end_deriv_1d(c, u, 0, cell, 1, 0));
    return (jl + jr) / (2.0 * c->hx);
  }
  const int nx = p->nx;
  int i = (int)(cell % nx), j = (int)(cell / nx);
  long nl = neighbour(p, i, j, 0, 0), nr = neighbour(p, i, j, 0, 1);
  long nb = neighbour(p, i, j, 1, 0), nt = neighbour(p, i, j, 1, 1);
  const double ghost = U(u, 0, 0, cell);
  double jv = 0.0, jh = 0.0;
  for (int cy = 0; cy <= 1; ++cy) {
    double gl = nl >= 0 ? corner_deriv_2d(c, u, 0, nl, 1, cy, 0, 0) : ghost;
    double gr = nr >= 0 ? corner_deriv_2d(c, u, 0, nr, 0, cy, 0, 0) : ghost;
    jv += 0.5 * fabs(corner_deriv_2d(c, u, 0, cell, 0, cy, 0, 0) - gl);
    jv += 0.5 * fabs(gr - corner_deriv_2d(c, u, 0, cell, 1, cy, 0, 0));
  }
  for (int cx = 0; cx <= 1; ++cx) {
    double gb = nb >= 0 ? corner_deriv_2d(c, u, 0, nb, cx, 1, 0, 0) : ghost;
    double gt = nt >= 0 ? corner_deriv_2d(c, u, 0, nt, cx, 0, 0, 0) : ghost;
    jh += 0.5 * fabs(corner_deriv_2d(c, u, 0, cell, cx, 0, 0, 0) - gb);
    jh += 0.5 * fabs(gt - corner_deriv_2d(c, u, 0, cell, cx, 1, 0, 0));
  }
  return jv / (2.0 * c->hx) + jh / (2.0 * c->hy);
}

void orc_jump_indicator(const orc_problem* p, const double* u, double* eta) {
  ctx_t c;
  make_ctx(p, &c);
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (long cell = 0; cell < c.ncell; ++cell) eta[cell] = eta_cell(p, &c, u, cell);
}

/* u^hyd of Algorithm 1 from the DG solution u (after the Runge-Kutta combination of a stage). */
void orc_hybrid(const orc_problem* p, const double* u, double dt, double* out) {
  ctx_t cc;
  make_ctx(p, &cc);
  const ctx_t* c = &cc;
  long n = orc_state_size(p);
  double* lim = (double*)malloc(sizeof(double) * n);
  double* eta = (double*)malloc(sizeof(double) * c->ncell);
  orc_filter(p, u, dt, lim);                           /* u^lim: the jump filter of u^DG */
  orc_jump_indicator(p, u, eta);
  double emax = 0.0;
  for (long cell = 0; cell < c->ncell; ++cell)
    if (eta[cell] > emax || isnan(eta[cell])) emax = eta[cell];
  for (long cell = 0; cell < c->ncell; ++cell) {
    const int troubled = eta[cell] > 1.0;
    const double w = troubled ? (emax - eta[cell]) / (emax - 1.0) : 1.0;
    for (int v = 0; v < c->nv; ++v)
      for (int m = 0; m < c->nm; ++m)
        U(out, v, m, cell) = troubled ? w * U(u, v, m, cell) + (1.0 - w) * U(lim, v, m, cell) : U(u, v, m, cell);
  }
  free(lim);
  free(eta);
}

/* ------------------------------------------------------------------------------------------ */
/* Positivity-preserving limiter of Zhang and Shu (J. Comput. Phys. 229, 2010), applied after the */
/* jump filter when the problem asks for it (the paper does so in Section 3.2).                   */
/* Checked at every point where the scheme evaluates the cell polynomial, the volume Gauss points */
/* and the Gauss points of the edges (1D: Gauss points and both ends), and at the rest of Zhang   */
/* and Shu's set: their positivity of the next averages rests on writing the average as a convex  */
/* combination of values at the tensor points of the Gauss rule and the N-point Gauss-Lobatto     */
/* rule with 2N - 3 >= k. For k = 2, 3 that is N = 3, whose interior node 0 adds the lines        */
/* xi = 0 and eta = 0 crossed with the Gauss nodes (1D: the point 0); for k = 2 they are volume   */
/* Gauss points already (0 is a node of the 3-point Gauss rule), for k = 3 they are new.         */
/* ------------------------------------------------------------------------------------------ */
#define ORC_MAXPP (ORC_MAXQ * ORC_MAXQ + 6 * ORC_MAXQ)
static int pp_points(const orc_problem* p, const ctx_t* c, double* xi, double* eta) {
  int n = 0;
  const int mid = p->k >= 2 && (c->nq % 2) == 0;   /* the Lobatto node 0 is not a Gauss node */
  if (p->dim == 1) {
    for (int a = 0; a < c->nq; ++a) { xi[n] = c->xq[a]; eta[n++] = 0.0; }
    xi[n] = -1.0; eta[n++] = 0.0;
    xi[n] = 1.0; eta[n++] = 0.0;
    if (mid) { xi[n] = 0.0; eta[n++] = 0.0; }
    return n;
  }
  for (int a = 0; a < c->nq; ++a)
    for (int b = 0; b < c->nq; ++b) { xi[n] = c->xq[a]; eta[n++] = c->xq[b]; }
  for (int g = 0; g < c->nq; ++g) {
    xi[n] = -1.0; eta[n++] = c->xq[g];
    xi[n] = 1.0; eta[n++] = c->xq[g];
    xi[n] = c->xq[g]; eta[n++] = -1.0;
    xi[n] = c->xq[g]; eta[n++] = 1.0;
  }
  if (mid)
    for (int g = 0; g < c->nq; ++g) {
      xi[n] = 0.0; eta[n++] = c->xq[g];
      xi[n] = c->xq[g]; eta[n++] = 0.0;
    }
  return n;
}

static void pp_cell(const orc_problem* p, const ctx_t* c, double* u, long cell) {
  double xi[ORC_MAXPP], eta[ORC_MAXPP];
  const int np = pp_points(p, c, xi, eta);
  double ubar[ORC_MAXNV];
  for (int v = 0; v < c->nv; ++v) ubar[v] = U(u, v, 0, cell);
  const double pbar = orc_pressure(p, ubar);
  /* admissibility margins relative to the cell average (the paper gives none): the density at
   * least eps_r = 1e-3 rho_bar, the pressure at least eps = min(1e-3 (rho_bar + |E_bar|), rho_bar,
   * p_bar); relative margins keep the velocity at a limited point bounded */
  const double eps_r = 1e-3 * ubar[0];
  double eps = 1e-3 * (ubar[0] + fabs(ubar[c->nv - 1]));
  if (ubar[0] < eps) eps = ubar[0];
  if (pbar < eps) eps = pbar;
  if (!(eps > 0.0) || !(eps_r > 0.0)) return;   /* inadmissible average: reported by the step */
  /* density: theta_1 = (rho_bar - eps_r) / (rho_bar - rho_min) when rho_min < eps_r */
  double rmin = ubar[0];
  for (int i = 0; i < np; ++i) {
    double val[ORC_MAXNV];
    eval_cell(p, c, u, cell, xi[i], eta[i], val);
    if (val[0] < rmin) rmin = val[0];
  }
  if (rmin < eps_r) {
    const double th1 = (ubar[0] - eps_r) / (ubar[0] - rmin);
    for (int m = 1; m < c->nm; ++m) U(u, 0, m, cell) *= th1;
  }
  /* pressure: theta_2 = min over points of t with p(u_bar + t (u(x) - u_bar)) = eps (bisection;
   * the admissible set is convex, so p - eps changes sign once on [0, 1]) */
  double th2 = 1.0;
  for (int i = 0; i < np; ++i) {
    double val[ORC_MAXNV];
    eval_cell(p, c, u, cell, xi[i], eta[i], val);
    if (orc_pressure(p, val) >= eps) continue;
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 60; ++it) {
      const double mid = 0.5 * (lo + hi);
      double w[ORC_MAXNV];
      for (int v = 0; v < c->nv; ++v) w[v] = ubar[v] + mid * (val[v] - ubar[v]);
      if (orc_pressure(p, w) >= eps) lo = mid; else hi = mid;
    }
    if (lo < th2) th2 = lo;
  }
  if (th2 < 1.0)
    for (int v = 0; v < c->nv; ++v)
      for (int m = 1; m < c->nm; ++m) U(u, v, m, cell) *= th2;
}

void orc_positivity(const orc_problem* p, double* u) {
  if (p->eq != ORC_EQ_EULER) return;
  ctx_t cc;
  make_ctx(p, &cc);
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (long cell = 0; cell < cc.ncell; ++cell) pp_cell(p, &cc, u, cell);
}

/* ------------------------------------------------------------------------------------------ */
/* Time stepping: third-order SSP Runge–Kutta in Shu–Osher form, Eq. (err_rk1), filter after   */
/* each stage, Eq. (err_rk2).                                                                 */
/* ------------------------------------------------------------------------------------------ */
static const double SO_C[3][3] = {{1.0, 0.0, 0.0}, {0.75, 0.25, 0.0}, {1.0 / 3.0, 0.0, 2.0 / 3.0}};
static const double SO_D[3][3] = {{1.0, 0.0, 0.0}, {0.0, 0.25, 0.0}, {0.0, 0.0, 2.0 / 3.0}};

/* Stage s (0,1,2): out = filter( c_s0 u^n + c_ss u^(s) + dt d_ss L(u^(s)) ). */
void orc_rk_stage(const orc_problem* p, int s, const double* un, const double* us, double dt,
                  double* out) {
  long n = orc_state_size(p);
  double* L = (double*)malloc(sizeof(double) * n);
  double* tmp = (double*)malloc(sizeof(double) * n);
  orc_residual(p, us, L);
  for (long e = 0; e < n; ++e) {
    double val = SO_C[s][s] * us[e] + dt * SO_D[s][s] * L[e];
    if (s > 0) val += SO_C[s][0] * un[e];
    tmp[e] = val;
  }
  if (p->filter) {
    double fdt = p->filter_dt_mode == 1 ? dt * SO_D[s][s] : dt;
    if (p->hybrid) orc_hybrid(p, tmp, fdt, out);   /* Algorithm 1 after every stage */
    else orc_filter(p, tmp, fdt, out);
  } else {
    memcpy(out, tmp, sizeof(double) * n);
  }
  if (p->positivity) orc_positivity(p, out);     /* after the filter (Section 3.2) */
  free(L);
  free(tmp);
}

int orc_check_physical(const orc_problem* p, const double* u) {
  ctx_t c;
  make_ctx(p, &c);
  for (long cell = 0; cell < c.ncell; ++cell) {
    double ubar[ORC_MAXNV];
    for (int v = 0; v < c.nv; ++v) {
      ubar[v] = u[((long)v * c.nm) * c.ncell + cell];
      if (!isfinite(ubar[v])) return -1;
    }
    if (p->eq == ORC_EQ_EULER && (ubar[0] <= 0.0 || orc_pressure(p, ubar) <= 0.0)) return -1;
  }
  return 0;
}

int orc_step(const orc_problem* p, double* u, double dt) {
  long n = orc_state_size(p);
  double* u1 = (double*)malloc(sizeof(double) * n);
  double* u2 = (double*)malloc(sizeof(double) * n);
  orc_rk_stage(p, 0, u, u, dt, u1);
  orc_rk_stage(p, 1, u, u1, dt, u2);
  orc_rk_stage(p, 2, u, u2, dt, u1);
  int bad = orc_check_physical(p, u1);
  if (!bad) memcpy(u, u1, sizeof(double) * n);
  free(u1);
  free(u2);
  return bad;
}

/* CFL rate from cell averages: 1D max_j beta_j / h; 2D max (beta^x/hx + beta^y/hy). With the
 * positivity-preserving limiter on, the wave speeds at the limiter's points count as well: Zhang
 * and Shu's positivity result for the cell averages needs the CFL bound on the largest of them. */
double orc_max_rate(const orc_problem* p, const double* u) {
  ctx_t c;
  make_ctx(p, &c);
  double best = 0.0;
  double xi[ORC_MAXPP], eta[ORC_MAXPP];
  const int np = (p->positivity && p->eq == ORC_EQ_EULER) ? pp_points(p, &c, xi, eta) : 0;
  for (long cell = 0; cell < c.ncell; ++cell) {
    double ubar[ORC_MAXNV];
    for (int v = 0; v < c.nv; ++v) ubar[v] = u[((long)v * c.nm) * c.ncell + cell];
    double r = orc_wave_speed(p, 0, ubar) / c.hx;
    if (p->dim == 2) r += orc_wave_speed(p, 1, ubar) / c.hy;
    if (r > best || isnan(r)) best = r;
    for (int i = 0; i < np; ++i) {
      double val[ORC_MAXNV];
      eval_cell(p, &c, u, cell, xi[i], eta[i], val);
      double rp = orc_wave_speed(p, 0, val) / c.hx;
      if (p->dim == 2) rp += orc_wave_speed(p, 1, val) / c.hy;
      if (rp > best || isnan(rp)) best = rp;
    }
  }
  return best;
}

/* dt = CFL / rate, clipped so that the last step lands on T. */
double orc_dt(const orc_problem* p, const double* u, double t, double T) {
  double dt = p->cfl / orc_max_rate(p, u);
  if (t + dt > T) dt = T - t;
  return dt;
}

int orc_advance(const orc_problem* p, double* u, double t0, double T, long max_steps,
                double* t_out, long* steps_out) {
  double t = t0;
  long steps = 0;
  int rc = 0;
  while (t < T && steps < max_steps) {
    double dtc = p->cfl / orc_max_rate(p, u);
    int last = (t + dtc >= T);
    double dt = last ? T - t : dtc;
    rc = orc_step(p, u, dt);
    if (rc) break;
    t = last ? T : t + dt;
    ++steps;
  }
  if (t_out) *t_out = t;
  if (steps_out) *steps_out = steps;
  return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Initial conditions and L2 projection                                                        */
/* ------------------------------------------------------------------------------------------ */
static void prim_to_cons(const orc_problem* p, const double* W, double* Uc) {
  double g = p->gamma;
  if (p->dim == 1) {
    double rho = W[0], vel = W[1], pr = W[2];
    Uc[0] = rho;
    Uc[1] = rho * vel;
    Uc[2] = pr / (g - 1.0) + 0.5 * rho * vel * vel;
    return;
  }
  double rho = W[0], vx = W[1], vy = W[2], pr = W[3];
  Uc[0] = rho;
  Uc[1] = rho * vx;
  Uc[2] = rho * vy;
  Uc[3] = pr / (g - 1.0) + 0.5 * rho * (vx * vx + vy * vy);
}

static int ic_value(const orc_problem* p, int ic, const double* prm, int nprm, double x, double y,
                    double* val) {
  if (ic == ORC_IC_SINE) {
    if (nprm < 4) return -1;
    double arg = prm[2] * (p->dim == 2 ? x + y : x) + prm[3];
    val[0] = prm[0] + prm[1] * sin(arg);
    return 0;
  }
  if (ic == ORC_IC_RIEMANN1D) {
    if (nprm < 7 || p->eq != ORC_EQ_EULER || p->dim != 1) return -1;
    prim_to_cons(p, x < prm[6] ? prm : prm + 3, val);
    return 0;
  }
  if (ic == ORC_IC_ENTROPY1D) {
    if (nprm < 5 || p->eq != ORC_EQ_EULER || p->dim != 1) return -1;
    double W[3] = {prm[0] + prm[1] * sin(prm[2] * x), prm[3], prm[4]};
    prim_to_cons(p, W, val);
    return 0;
  }
  if (ic == ORC_IC_QUADRANT2D) {
    if (nprm < 18 || p->eq != ORC_EQ_EULER || p->dim != 2) return -1;
    double xs = prm[16], ys = prm[17];
    int qd = (x > xs) ? (y > ys ? 0 : 3) : (y > ys ? 1 : 2);   /* Q1..Q4 */
    prim_to_cons(p, prm + 4 * qd, val);
    return 0;
  }
  if (ic == ORC_IC_VORTEX2D) {
    if (nprm < 4 || p->eq != ORC_EQ_EULER || p->dim != 2) return -1;
    double W[4];
    orc_vortex_exact(p->gamma, prm[0], prm[1], prm[2], p->x1 - p->x0, p->y1 - p->y0, p->x0, p->y0,
                     x, y, prm[3], W);
    prim_to_cons(p, W, val);
    return 0;
  }
  if (ic == ORC_IC_COEFFS_ZERO) {
    for (int v = 0; v < orc_nvars(p); ++v) val[v] = 0.0;
    return 0;
  }
  return -1;
}

/* u^l = (int u0 P_l) / (int P_l^2) per cell (tensor product in 2D), Gauss rule with nq_init points. */
int orc_project(const orc_problem* p, int ic, const double* prm, int nprm, int nq_init, double* u) {
  ctx_t cc;
  make_ctx(p, &cc);
  const ctx_t* c = &cc;
  int nq = nq_init > 0 ? nq_init : p->k + 3;
  if (nq > ORC_MAXQ) return -1;
  double xq[ORC_MAXQ], wq[ORC_MAXQ];
  orc_gauss(nq, xq, wq);
  double probe[ORC_MAXNV];
  if (ic_value(p, ic, prm, nprm, p->x0, p->y0, probe)) return -1;
  const int nx = p->nx;
  for (long cell = 0; cell < c->ncell; ++cell) {
    int i = (int)(cell % nx), j = (int)(cell / nx);
    double xc = p->x0 + (i + 0.5) * c->hx, yc = p->dim == 2 ? p->y0 + (j + 0.5) * c->hy : 0.0;
    double acc[ORC_MAXNV][ORC_MAXNM];
    memset(acc, 0, sizeof(acc));
    int nb = p->dim == 2 ? nq : 1;
    for (int a = 0; a < nq; ++a)
      for (int b = 0; b < nb; ++b) {
        double x = xc + 0.5 * c->hx * xq[a];
        double y = p->dim == 2 ? yc + 0.5 * c->hy * xq[b] : 0.0;
        double val[ORC_MAXNV];
        ic_value(p, ic, prm, nprm, x, y, val);
        double w = wq[a] * (p->dim == 2 ? wq[b] : 1.0);
        for (int m = 0; m < c->nm; ++m) {
          double phi = orc_legendre(c->mp[m], xq[a]) * (p->dim == 2 ? orc_legendre(c->mq[m], xq[b]) : 1.0);
          for (int v = 0; v < c->nv; ++v) acc[v][m] += w * val[v] * phi;
        }
      }
    for (int m = 0; m < c->nm; ++m) {
      double nrm = c->nrm[c->mp[m]] * (p->dim == 2 ? c->nrm[c->mq[m]] : 1.0);
      for (int v = 0; v < c->nv; ++v) U(u, v, m, cell) = acc[v][m] / nrm;
    }
  }
  return 0;
}
