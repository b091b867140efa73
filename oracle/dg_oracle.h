/*
 * dg_oracle.h — plain, slow FP64 CPU oracle for the Runge–Kutta DG method with the jump filter
 * (Wei, Zhou & Xia, "The jump filter in the discontinuous Galerkin method for hyperbolic
 * conservation laws", arXiv 2407.19169).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load this code: only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg use it. It shares no source,
 * header, table or helper with the CUDA library.
 *
 * It follows the paper's steps in the paper's order and notation:
 *   - Section 2.1, Eq. (scheme:DG): semi-discrete modal DG in 1D with a two-point numerical flux;
 *   - Eq. (GLbasisequation): Legendre basis on the reference cell [-1,1];
 *   - Eqs. (para:damp2)-(para:damp21), (timespli:1dscalar): the mode-dependent jump filter;
 *   - Section 2.3, Eqs. (para:dampsystems1d)-(timespli:sys): systems take the max over components;
 *   - Section 2.2, Eqs. (para:2ddamp), (para:damp22d)-(para:damp22d1): the 2D filter with the
 *     trapezoidal rule for edge-averaged jumps;
 *   - Eqs. (rkdg1), (err_rk1)-(err_rk2): Shu–Osher Runge–Kutta with the filter after every stage;
 *   - Section 3: local Lax–Friedrichs flux, third-order SSP Runge–Kutta; Euler parameters
 *     c_f^l = beta/(4 l(l+1)) / Hbar (1D) and (c_fx, c_fy) = (h_y beta^x, h_x beta^y)/(4 lambda Hbar) (2D).
 *
 * Canonical state layout (shared with the C ABI by specification only): u[(v*NM + m)*ncell + c],
 * FP64, standard Legendre P_l(1)=1. 1D: c = i. 2D: c = i + nx*j, mode m enumerates (p,q) with q the
 * outer and p the inner index (Q^k: m = p + (k+1) q; P^k: the same order, skipping p+q > k).
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXK 4         /* highest polynomial degree the oracle supports */
#define ORC_MAXQ 12        /* highest Gauss rule order */
#define ORC_MAXNV 4
#define ORC_MAXNM ((ORC_MAXK + 1) * (ORC_MAXK + 1))

enum { ORC_EQ_ADVECTION = 0, ORC_EQ_BURGERS = 1, ORC_EQ_EULER = 2 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_OUTFLOW = 1 };
enum { ORC_BASIS_Q = 0, ORC_BASIS_P = 1 };
/* Damping of the filter (Section 2.1):
 *   ORC_FILTER_JUMP   the mode-dependent jump filter, Eqs. (para:damp2)-(para:damp21) (the paper's scheme)
 *   ORC_FILTER_GLOBAL one damping coefficient for all modes, Eq. (para:damp): sigma_j from the jumps of
 *                     every derivative order, sigma_j^l = sigma_j (2/h)^2 l(l+1), c_f = c_f^l
 *   ORC_FILTER_OEDG   the OEDG damping as the paper writes it in its notation:
 *                     sigma^{l,OE} = c_f^OE (h ||[u]|| + sum_{m=1..l} (2m+1)/m! h^{m+1} ||[d^m u]||) / h^2,
 *                     c_f^OE = beta / (2 (2k-1) ||u - avg(u)||_{L^inf(Omega)}) (0 if u = avg(u)) */
enum { ORC_FILTER_JUMP = 0, ORC_FILTER_GLOBAL = 1, ORC_FILTER_OEDG = 2 };

/* Initial-condition kinds for the L2 projection (Section 3 examples and synthetic workloads). */
enum {
  ORC_IC_SINE = 0,        /* scalar: a + b*sin(w*(x + y) + phi)       params: a, b, w, phi      */
  ORC_IC_RIEMANN1D = 1,   /* Euler 1D: rhoL,uL,pL, rhoR,uR,pR, xs     (primitive states)       */
  ORC_IC_ENTROPY1D = 2,   /* Euler 1D: rho=r0+A sin(w x), u=u0, p=p0  params: r0, A, w, u0, p0 */
  ORC_IC_QUADRANT2D = 3,  /* Euler 2D: 4 states (rho,u,v,p) Q1..Q4, then xs, ys               */
  ORC_IC_VORTEX2D = 4,    /* Euler 2D: isentropic vortex of Example 3.4(a); x0, y0, beta, t    */
  ORC_IC_COEFFS_ZERO = 5  /* zero state (for tests that fill coefficients by hand)            */
};

typedef struct {
  int dim;                 /* 1 or 2 */
  int nx, ny;              /* cells per direction (ny = 1 in 1D) */
  double x0, x1, y0, y1;   /* domain */
  int bc[4];               /* x-low, x-high, y-low, y-high: ORC_BC_* */
  int k;                   /* polynomial degree */
  int basis;               /* 2D only: ORC_BASIS_Q (tensor product) or ORC_BASIS_P (total degree) */
  int eq;                  /* ORC_EQ_* */
  double gamma;            /* Euler ratio of specific heats */
  double adv[2];           /* linear advection velocity */
  int filter;              /* 1 = jump filter after every stage, 0 = plain RKDG */
  double cfl;              /* CFL number */
  int nq;                  /* Gauss points per direction for volume and edges (0 -> k+1) */
  int filter_dt_mode;      /* 0: exp(-sigma*dt) with the full step dt after every stage;
                              1: the stage's own effective step (dt, dt/4, 2dt/3) */
  int positivity;          /* Euler: 1 = Zhang-Shu positivity-preserving limiter after the filter */
  int hybrid;              /* 1 = hybrid limiter of Algorithm 1 (jump filter as the low-order part) */
  int filter_kind;         /* ORC_FILTER_*: the damping coefficients of the filter */
  int filter_study;        /* 2D jump filter, other readings for a study (0 = the readings in use):
                              bit 0: beta^x, beta^y as the largest |u|+c, |v|+c over the cell's
                                     volume and edge Gauss points instead of at the average;
                              bit 1: Hbar as the cell average of H(u(x)) (volume Gauss rule)
                                     instead of H of the average state;
                              bit 2: the max over components taken per direction and the two
                                     directions added, instead of the max of the sum */
} orc_problem;

/* ---- basis (orc_basis.c) ---- */
double orc_legendre(int n, double x);                          /* P_n(x) by Bonnet's recurrence */
double orc_legendre_deriv(int n, int m, double x);             /* d^m/dx^m P_n(x), monomial form  */
int    orc_gauss(int n, double* x, double* w);                 /* Gauss–Legendre on [-1,1], Newton */
double orc_legendre_norm(int n);                               /* int_{-1}^{1} P_n^2, by quadrature */

/* ---- physics (orc_physics.c) ---- */
int    orc_nvars(const orc_problem* p);
void   orc_flux(const orc_problem* p, int dir, const double* u, double* f);
double orc_wave_speed(const orc_problem* p, int dir, const double* u);
double orc_enthalpy(const orc_problem* p, const double* u);
double orc_pressure(const orc_problem* p, const double* u);

/* ---- DG operator, filter and time stepping (orc_dg.c) ---- */
int    orc_nmodes(const orc_problem* p);
void   orc_mode_pq(const orc_problem* p, int m, int* pdeg, int* qdeg);
long   orc_state_size(const orc_problem* p);
int    orc_project(const orc_problem* p, int ic, const double* prm, int nprm, int nq_init, double* u);
double orc_max_rate(const orc_problem* p, const double* u);   /* 1D: max beta/h; 2D: max beta^x/hx+beta^y/hy */
double orc_dt(const orc_problem* p, const double* u, double t, double T);
void   orc_residual(const orc_problem* p, const double* u, double* R);
void   orc_filter(const orc_problem* p, const double* u, double dt, double* out);
void   orc_positivity(const orc_problem* p, double* u);            /* Zhang-Shu limiter, in place */
void   orc_jump_indicator(const orc_problem* p, const double* u, double* eta); /* Algorithm 1 eta_j */
void   orc_hybrid(const orc_problem* p, const double* u, double dt, double* out);  /* Algorithm 1 */
void   orc_filter_sigma(const orc_problem* p, const double* u, double* sigma); /* sigma^l per cell, l=0..lmax */
void   orc_oedg_norms(const orc_problem* p, const double* u, double* ninf);   /* ||u_v - avg u_v||_inf */
void   orc_rk_stage(const orc_problem* p, int s, const double* un, const double* us, double dt, double* out);
int    orc_step(const orc_problem* p, double* u, double dt);  /* one SSP-RK3 step in place; 0 = ok */
int    orc_advance(const orc_problem* p, double* u, double t0, double T, long max_steps,
                   double* t_out, long* steps_out);
int    orc_check_physical(const orc_problem* p, const double* u);  /* 0 ok, -1 non-physical average */

/* ---- diagnostics and exact solutions (orc_exact.c) ---- */
void   orc_mass(const orc_problem* p, const double* u, double* mass);      /* per variable */
double orc_energy(const orc_problem* p, const double* u);                  /* sum of L2 norms^2 */
double orc_burgers_exact(double x, double t, double a, double b, double w, double phi, double L);
int    orc_riemann_exact(double gamma, const double* WL, const double* WR, double xi, double* W);
void   orc_vortex_exact(double gamma, double x0, double y0, double beta, double Lx, double Ly,
                        double xlo, double ylo, double x, double y, double t, double* W);
int    orc_errors(const orc_problem* p, const double* u, int exact_kind, const double* prm, int nprm,
                  double t, int nq_err, int var, double* l1, double* l2, double* linf);
void   orc_eval(const orc_problem* p, const double* u, int cell, double xi, double eta, double* val);
void   orc_set_threads(int n);
int    orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
