/*
 * orc_physics.c — fluxes, wave speeds and enthalpy for the FP64 oracle.
 * TEST INFRASTRUCTURE ONLY (see dg_oracle.h).
 *
 *   scalar law   u_t + f(u)_x = 0                     (Eq. eqn:scl)
 *     linear advection f = c u;  Burgers f = u^2/2    (Example 3.1)
 *   1D Euler     U = (rho, m, E), F = (m, m^2/rho + p, m/rho (E + p)),  p = (gamma-1)(E - m^2/(2 rho))
 *   2D Euler     U = (rho, mx, my, E), F = (m^T, rho u u^T + p I, (E + p) u^T)   (Section 3.2)
 *   H = (E + p)/rho (Section 3.1); beta = spectral radius of dF/dU: |u_n| + c, c = sqrt(gamma p / rho).
 */
#include "dg_oracle.h"
#include <math.h>

int orc_nvars(const orc_problem* p) {
  if (p->eq == ORC_EQ_EULER) return p->dim == 1 ? 3 : 4;
  return 1;
}

double orc_pressure(const orc_problem* p, const double* u) {
  if (p->eq != ORC_EQ_EULER) return 0.0;
  double rho = u[0];
  if (p->dim == 1) {
    double m = u[1], E = u[2];
    return (p->gamma - 1.0) * (E - 0.5 * m * m / rho);
  }
  double mx = u[1], my = u[2], E = u[3];
  return (p->gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho);
}

/* Flux component in direction dir (0 = x, 1 = y). */
void orc_flux(const orc_problem* p, int dir, const double* u, double* f) {
  if (p->eq == ORC_EQ_ADVECTION) { f[0] = p->adv[dir] * u[0]; return; }
  if (p->eq == ORC_EQ_BURGERS) { f[0] = 0.5 * u[0] * u[0]; return; }
  double rho = u[0];
  double pr = orc_pressure(p, u);
  if (p->dim == 1) {
    double m = u[1], E = u[2], vel = m / rho;
    f[0] = m;
    f[1] = m * vel + pr;
    f[2] = vel * (E + pr);
    return;
  }
  double mx = u[1], my = u[2], E = u[3];
  double vx = mx / rho, vy = my / rho;
  double vn = dir == 0 ? vx : vy;
  f[0] = rho * vn;
  f[1] = mx * vn + (dir == 0 ? pr : 0.0);
  f[2] = my * vn + (dir == 1 ? pr : 0.0);
  f[3] = vn * (E + pr);
}

/* Spectral radius of the flux Jacobian in direction dir. */
double orc_wave_speed(const orc_problem* p, int dir, const double* u) {
  if (p->eq == ORC_EQ_ADVECTION) return fabs(p->adv[dir]);
  if (p->eq == ORC_EQ_BURGERS) return fabs(u[0]);
  double rho = u[0];
  double pr = orc_pressure(p, u);
  double c = sqrt(p->gamma * pr / rho);
  double vn = (p->dim == 1) ? u[1] / rho : u[1 + dir] / rho;
  return fabs(vn) + c;
}

/* Enthalpy H = (E + p)/rho for Euler; scalar laws use 1 (no 1/H factor in c_f). */
double orc_enthalpy(const orc_problem* p, const double* u) {
  if (p->eq != ORC_EQ_EULER) return 1.0;
  double E = (p->dim == 1) ? u[2] : u[3];
  return (E + orc_pressure(p, u)) / u[0];
}
