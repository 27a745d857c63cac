/*
 * sph_oracle.c -- FP64 CPU oracle of the macroscale SPH step (2D) of the
 * LHMM: summation density, Tait pressure (Eq. tait), the Espanol-Revenga
 * momentum equation with the micro-to-macro stress term (Eq.
 * sph_continuity), velocity-Verlet, and the SPH velocity gradient that is
 * sent down to the micro-domains (Eq. macro_micro).
 *
 * TEST INFRASTRUCTURE ONLY (see lhmm_oracle.h).  O(N^2) pair search with the
 * minimum image: obviously correct, slow.
 *
 * Readings of the paper used here:
 *  S1 kernel: Wendland C2 in 2D with support radius h (default), or the Lucy
 *     kernel of Appendix A; F_IJ = -W'(r)/r.
 *  S2 d_I includes the self term W(0).
 *  S3 viscous coefficients: a = 2 eta_s - zeta_s, b = 4 zeta_s reproduce a
 *     2D shear viscosity eta_s in the continuum limit; the printed
 *     b = 4 zeta_s + 2 eta_s is kept as an option (it yields 1.25 eta_s).
 *  S4 velocity gradient with the volume factor 1/d_J that Eq. macro_micro
 *     omits: L_ab = dv_a/dx_b = sum_J (F_IJ/d_J) v_IJ,a r_IJ,b.
 *  S5 background pressure p_b = theta c^2 rho0 / 7.
 *  S6 body force per unit mass; reverse Poiseuille: +F for y >= Ly/2 and
 *     -F below (Sec. 6.1).
 *  S7 wall particles are fixed (v = 0), enter density, pressure and viscous
 *     sums as neighbours, and carry no micro stress.
 */
#include "lhmm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

double orc_sph_W(int kernel, double r, double h) {
  double q = r / h;
  if (q >= 1.0) return 0.0;
  double omq = 1.0 - q;
  if (kernel == ORC_KERNEL_LUCY)
    return 5.0 / (M_PI * h * h) * (1.0 + 3.0 * q) * omq * omq * omq;
  return 7.0 / (M_PI * h * h) * (1.0 + 4.0 * q) * omq * omq * omq * omq;
}

/* F(r) = -W'(r)/r, from differentiating the two kernels above */
double orc_sph_F(int kernel, double r, double h) {
  double q = r / h;
  if (q >= 1.0) return 0.0;
  double omq = 1.0 - q;
  double h4 = h * h * h * h;
  if (kernel == ORC_KERNEL_LUCY) return 60.0 / (M_PI * h4) * omq * omq;
  return 140.0 / (M_PI * h4) * omq * omq * omq;
}

double orc_sph_pressure(const orc_sph_params* p, double rho) {
  double pb = p->theta_pb * p->c * p->c * p->rho0 / 7.0;
  return p->c * p->c * p->rho0 / 7.0 * (pow(rho / p->rho0, 7.0) - 1.0) + pb;
}

static void min_image2(const orc_sph_params* p, const double* pos, int I, int J, double d[2]) {
  d[0] = pos[2 * I] - pos[2 * J];
  d[1] = pos[2 * I + 1] - pos[2 * J + 1];
  d[0] -= p->Lx * nearbyint(d[0] / p->Lx);
  d[1] -= p->Ly * nearbyint(d[1] / p->Ly);
}

void orc_sph_density(const orc_sph_params* p, const double* pos, double* d) {
  for (int I = 0; I < p->n; ++I) {
    double s = 0.0;
    for (int J = 0; J < p->n; ++J) {
      double r[2];
      min_image2(p, pos, I, J, r);
      s += orc_sph_W(p->kernel, sqrt(r[0] * r[0] + r[1] * r[1]), p->h);
    }
    d[I] = s;
  }
}

static void visc_coeffs(const orc_sph_params* p, double* a, double* b) {
  *a = 2.0 * p->eta_s - p->zeta_s;
  *b = (p->visc_coeffs == ORC_VISC_PAPER_LITERAL) ? 4.0 * p->zeta_s + 2.0 * p->eta_s
                                                  : 4.0 * p->zeta_s;
}

void orc_sph_accel(const orc_sph_params* p, const double* pos, const double* vel,
                   const int* is_wall, const double* stress3, double* acc, double* d_out) {
  const int n = p->n;
  double* d = (double*)malloc(sizeof(double) * n);
  double* pr = (double*)malloc(sizeof(double) * n);
  orc_sph_density(p, pos, d);
  for (int I = 0; I < n; ++I) pr[I] = orc_sph_pressure(p, p->mass * d[I]);
  double a, b;
  visc_coeffs(p, &a, &b);
  for (int I = 0; I < n; ++I) {
    acc[2 * I] = acc[2 * I + 1] = 0.0;
    if (is_wall && is_wall[I]) continue;
    double f[2] = {0.0, 0.0};
    for (int J = 0; J < n; ++J) {
      if (J == I) continue;
      double r[2];
      min_image2(p, pos, I, J, r);
      double rr = sqrt(r[0] * r[0] + r[1] * r[1]);
      double F = orc_sph_F(p->kernel, rr, p->h);
      if (F == 0.0) continue;
      double e[2] = {r[0] / rr, r[1] / rr};
      double v[2] = {vel[2 * I] - vel[2 * J], vel[2 * I + 1] - vel[2 * J + 1]};
      /* pressure term */
      double P = pr[I] / (d[I] * d[I]) + pr[J] / (d[J] * d[J]);
      f[0] += P * F * r[0];
      f[1] += P * F * r[1];
      /* viscous term */
      double ve = v[0] * e[0] + v[1] * e[1];
      double cv = F / (d[I] * d[J]);
      f[0] -= (a * v[0] + b * ve * e[0]) * cv;
      f[1] -= (a * v[1] + b * ve * e[1]) * cv;
      /* micro-to-macro coupling term: <pi>_IJ = pi_I/d_I^2 + pi_J/d_J^2 */
      if (stress3) {
        double sI[3] = {0, 0, 0}, sJ[3] = {0, 0, 0};
        if (!(is_wall && is_wall[I])) { sI[0] = stress3[3 * I]; sI[1] = stress3[3 * I + 1]; sI[2] = stress3[3 * I + 2]; }
        if (!(is_wall && is_wall[J])) { sJ[0] = stress3[3 * J]; sJ[1] = stress3[3 * J + 1]; sJ[2] = stress3[3 * J + 2]; }
        double xx = sI[0] / (d[I] * d[I]) + sJ[0] / (d[J] * d[J]);
        double xy = sI[1] / (d[I] * d[I]) + sJ[1] / (d[J] * d[J]);
        double yy = sI[2] / (d[I] * d[I]) + sJ[2] / (d[J] * d[J]);
        f[0] -= (xx * r[0] + xy * r[1]) * F;
        f[1] -= (xy * r[0] + yy * r[1]) * F;
      }
    }
    double g[2] = {p->body_force[0], p->body_force[1]};
    if (p->body_mode == ORC_BODY_REVERSE_POISEUILLE) {
      g[0] = (pos[2 * I + 1] >= 0.5 * p->Ly) ? p->body_force[0] : -p->body_force[0];
      g[1] = 0.0;
    }
    acc[2 * I] = f[0] / p->mass + g[0];
    acc[2 * I + 1] = f[1] / p->mass + g[1];
  }
  if (d_out) memcpy(d_out, d, sizeof(double) * n);
  free(d);
  free(pr);
}

void orc_sph_velgrad(const orc_sph_params* p, const double* pos, const double* vel,
                     const double* d, double* L4) {
  for (int I = 0; I < p->n; ++I) {
    double Lxx = 0, Lxy = 0, Lyx = 0, Lyy = 0;
    for (int J = 0; J < p->n; ++J) {
      if (J == I) continue;
      double r[2];
      min_image2(p, pos, I, J, r);
      double rr = sqrt(r[0] * r[0] + r[1] * r[1]);
      double F = orc_sph_F(p->kernel, rr, p->h);
      if (F == 0.0) continue;
      double v[2] = {vel[2 * I] - vel[2 * J], vel[2 * I + 1] - vel[2 * J + 1]};
      double c = F / d[J];
      Lxx += c * v[0] * r[0];
      Lxy += c * v[0] * r[1];
      Lyx += c * v[1] * r[0];
      Lyy += c * v[1] * r[1];
    }
    L4[4 * I] = Lxx; L4[4 * I + 1] = Lxy; L4[4 * I + 2] = Lyx; L4[4 * I + 3] = Lyy;
  }
}

void orc_sph_steps(const orc_sph_params* p, double* pos, double* vel, double* acc,
                   const int* is_wall, const double* stress3, int n_sub) {
  const int n = p->n;
  const double dt = p->dt;
  for (int s = 0; s < n_sub; ++s) {
    for (int I = 0; I < n; ++I) {
      if (is_wall && is_wall[I]) continue;
      vel[2 * I] += 0.5 * dt * acc[2 * I];
      vel[2 * I + 1] += 0.5 * dt * acc[2 * I + 1];
      pos[2 * I] += dt * vel[2 * I];
      pos[2 * I + 1] += dt * vel[2 * I + 1];
      pos[2 * I] -= p->Lx * floor(pos[2 * I] / p->Lx);
      pos[2 * I + 1] -= p->Ly * floor(pos[2 * I + 1] / p->Ly);
    }
    orc_sph_accel(p, pos, vel, is_wall, stress3, acc, NULL);
    for (int I = 0; I < n; ++I) {
      if (is_wall && is_wall[I]) continue;
      vel[2 * I] += 0.5 * dt * acc[2 * I];
      vel[2 * I + 1] += 0.5 * dt * acc[2 * I + 1];
    }
  }
}
