/*
 * micro_oracle.c -- FP64 CPU oracle of one LHMM micro-domain step
 * (DPD + FENE + velocity-Verlet + imposed flow + Irving-Kirkwood stress).
 *
 * TEST INFRASTRUCTURE ONLY (see lhmm_oracle.h).  Plain loops, double
 * precision, no blocking or fusion beyond what the equations state.
 *
 * Readings of the paper used here:
 *  R1 weight functions: w^R(r) = 1 - r/rc, w^D = (w^R)^2 (FDT, Sec. 2.3);
 *     the paper names the FDT relation but never prints w^R.
 *  R2 random force: F^R = sigma w^R theta_ij e_ij / sqrt(dt); the 1/sqrt(dt)
 *     of the time-discretised Wiener increment is missing from Eq. random.
 *  R3 theta_ij: Philox4x32-10 (Salmon et al., SC'11) keyed by (low seed word,
 *     high seed word xor box) and counted by (min id, max id, step); Box-Muller on the top 23 bits of
 *     the first two output words, so theta_ij = theta_ji.
 *  R4 FENE: attractive, F_i = -H r_ij / (1 - (r/R0)^2); Eq. fene_force drops
 *     the minus sign that its commented -grad U states.
 *  R5 the DPD sum of Eq. F_DPD runs over all j != i, bonded pairs included
 *     (alternatives: exclude pairs of one chain up to K bonds apart, as a
 *     LAMMPS special_bonds setting does).
 *  R6 velocity-Verlet in the LAMMPS form named by the coupling protocol:
 *     half kick, drift, forces (dissipative term with half-step v), half kick.
 *  R7 Lees-Edwards sliding-brick images for steady shear du_x/dy.
 *  R8 AFBC: concentric cubic shells by fraction of the edge (Table 2), region
 *     by max-norm distance from the box centre; after the second half kick
 *     every BC bead gets v = L r' (Eq. micro_bc), r' relative to the centre.
 *     Alternative (afbc_mode = 1): v = L r' + (v - mean of the BC beads of
 *     the bead's cell), keeping the thermal motion of the shell.
 *  R9 IK: uniform weight w_IK = 1/V_core on the core; the bond function is
 *     the length fraction of segment i->j inside the core over V_core.
 *     Sign: pi = -(sum m dv(x)dv + sum_{i<j} F_ij (x) r_ij)/V_core, i.e.
 *     f_ij of Eq. potential_stress is the force on j due to i.
 *  R10 a bond at |r| >= R0 (Eq. fene_force undefined) is reported; its
 *     stiffness is held at the (r/R0)^2 = 0.99 value so the run continues.
 *  R11 the paper's melt boxes are 2D (number density per area, Table 1):
 *     dim = 2 keeps z = 0, one cell layer, pairs in the plane only, AFBC
 *     squares, and the IK stress per core area.
 */
#include "lhmm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random   */
/* numbers: as easy as 1, 2, 3").  Multipliers and Weyl key increments  */
/* are the published constants of the method.                           */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = M0 * (uint64_t)x0;
    uint64_t p1 = M1 * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* R3: two uniforms u = (k + 1/2) 2^-23 from the top 23 bits k of a word
 * (exactly representable in any binary float with a >= 24-bit significand,
 * so every precision draws the same u), then Box-Muller. */
double orc_theta_from_words(uint32_t x0, uint32_t x1) {
  const double two_m23 = 1.0 / 8388608.0;
  double u1 = ((double)(x0 >> 9) + 0.5) * two_m23;
  double u2 = ((double)(x1 >> 9) + 0.5) * two_m23;
  return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

double orc_pair_theta(uint64_t seed, int box_id, int id_i, int id_j, uint64_t step) {
  uint32_t key[2], ctr[4], out[4];
  key[0] = (uint32_t)seed;
  key[1] = (uint32_t)(seed >> 32) ^ (uint32_t)box_id;
  ctr[0] = (uint32_t)(id_i < id_j ? id_i : id_j);
  ctr[1] = (uint32_t)(id_i < id_j ? id_j : id_i);
  ctr[2] = (uint32_t)step;
  ctr[3] = (uint32_t)(step >> 32);
  orc_philox4x32_10(ctr, key, out);
  return orc_theta_from_words(out[0], out[1]);
}

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */
static double wrap_to(double x, double L) { /* into [0, L) */
  double y = x - L * floor(x / L);
  if (y >= L) y -= L;
  if (y < 0) y += L;
  return y;
}

/* minimum-image displacement r_ij = r_i - r_j and v_ij, with Lees-Edwards
 * images in y for shear rate gdot (R7). */
static void pair_disp(const orc_dpd_params* p, const orc_box* b, double gdot, int i, int j,
                      double dr[3], double dv[3]) {
  const double Lx = b->edge[0], Ly = b->edge[1], Lz = b->edge[2];
  for (int a = 0; a < 3; ++a) {
    dr[a] = b->pos[3 * i + a] - b->pos[3 * j + a];
    dv[a] = b->vel[3 * i + a] - b->vel[3 * j + a];
  }
  if (p->flow_mode == ORC_FLOW_LEES_EDWARDS) {
    if (dr[1] > 0.5 * Ly) {          /* j taken as its image above the box */
      dr[1] -= Ly; dr[0] -= b->le_offset; dv[0] -= gdot * Ly;
    } else if (dr[1] < -0.5 * Ly) {  /* j taken as its image below the box */
      dr[1] += Ly; dr[0] += b->le_offset; dv[0] += gdot * Ly;
    }
  } else {
    dr[1] -= Ly * nearbyint(dr[1] / Ly);
  }
  dr[0] -= Lx * nearbyint(dr[0] / Lx);
  dr[2] -= Lz * nearbyint(dr[2] / Lz);
}

int orc_afbc_region(const orc_dpd_params* p, const double edge[3], const double r[3]) {
  int core = 1, bc = 1;
  for (int a = 0; a < (p->dim == 2 ? 2 : 3); ++a) {
    double x = fabs(r[a] - 0.5 * edge[a]);
    if (!(x < 0.5 * p->core_frac * edge[a])) core = 0;
    if (!(x < (0.5 * p->core_frac + p->bc_frac) * edge[a])) bc = 0;
  }
  return core ? 0 : (bc ? 1 : 2);
}

/* Length fraction of the segment a->b lying in the open box |x_k| < half[k]
 * (R9: the IK bond function for a uniform weight, times V_core).  Each axis
 * restricts the segment parameter s in [0,1] to an interval. */
double orc_segment_fraction(const double a[3], const double b[3], const double half[3]) {
  double lo = 0.0, hi = 1.0;
  for (int k = 0; k < 3; ++k) {
    double d = b[k] - a[k];
    if (d == 0.0) {
      if (!(fabs(a[k]) < half[k])) return 0.0;
      continue;
    }
    double s1 = (-half[k] - a[k]) / d, s2 = (half[k] - a[k]) / d;
    double smin = s1 < s2 ? s1 : s2, smax = s1 < s2 ? s2 : s1;
    if (smin > lo) lo = smin;
    if (smax < hi) hi = smax;
  }
  return hi > lo ? hi - lo : 0.0;
}

/* volume (area in 2D) over which the IK stress averages (R9) */
static double core_volume(const orc_dpd_params* p, const orc_box* b) {
  const int d = p->dim == 2 ? 2 : 3;
  double v = 1.0;
  for (int a = 0; a < d; ++a)
    v *= (p->flow_mode == ORC_FLOW_AFBC ? p->core_frac : 1.0) * b->edge[a];
  return v;
}

/* pair (i, j) excluded from the DPD sum: same chain, at most K bonds apart,
 * K = max(exclude_bonds, 1 if dpd_on_bonded = 0) (R5 and its alternatives) */
static int excluded(const orc_dpd_params* p, const orc_box* b, int i, int j) {
  int K = p->exclude_bonds > 0 ? p->exclude_bonds : 0;
  if (!p->dpd_on_bonded && K < 1) K = 1;
  int lo = i < j ? i : j, hi = i < j ? j : i, d = hi - lo;
  if (d < 1 || d > K) return 0;
  if (hi >= b->n_chains * b->chain_len) return 0;
  return (lo % b->chain_len) + d < b->chain_len; /* same chain */
}

/* ------------------------------------------------------------------ */
/* forces                                                              */
/* ------------------------------------------------------------------ */
/* F_ij on i from j by Eqs. conservative, dissipative, random (R1, R2). */
static void dpd_pair_force(const orc_dpd_params* p, const orc_box* b, int i, int j,
                           const double dr[3], const double dv[3], double F[3], int* hit) {
  double r2 = dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2];
  F[0] = F[1] = F[2] = 0.0;
  *hit = 0;
  if (!(r2 < p->rc * p->rc) || r2 == 0.0) return;
  double r = sqrt(r2);
  double e[3] = {dr[0] / r, dr[1] / r, dr[2] / r};
  double wR = 1.0 - r / p->rc;
  double wD = wR * wR;
  double ev = e[0] * dv[0] + e[1] * dv[1] + e[2] * dv[2];
  double theta = orc_pair_theta(p->seed, b->box_id, i, j, b->step);
  double fC = p->a_ij * wR;
  double fD = -p->gamma * wD * ev;
  double fR = p->sigma * wR * theta / sqrt(p->dt);
  double f = fC + fD + fR;
  F[0] = f * e[0]; F[1] = f * e[1]; F[2] = f * e[2];
  *hit = 1;
}

/* Eq. fene_force with the attractive sign (R4). Returns nonzero on |r| >= R0,
 * where the spring is undefined; the run then continues with the spring
 * stiffness held at its (r/R0)^2 = 0.99 value (R10) and the error reported. */
static int fene_force(const orc_dpd_params* p, const double dr[3], double F[3]) {
  double r2 = dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2];
  double x = r2 / (p->R0 * p->R0);
  int over = 0;
  if (!(x < 1.0)) { x = 0.99; over = 1; }
  double c = -p->H_fene / (1.0 - x);
  F[0] = c * dr[0]; F[1] = c * dr[1]; F[2] = c * dr[2];
  return over;
}

static double lees_edwards_rate(const orc_dpd_params* p, const double L[9]) {
  return p->lambda_star * L[1]; /* du_x/dy */
}

/* position relative to the box centre of bead i */
static void rel_pos(const orc_box* b, int i, double rp[3]) {
  for (int a = 0; a < 3; ++a) rp[a] = b->pos[3 * i + a] - 0.5 * b->edge[a];
}

/* bond-function weight (times V_core) of pair (i, j) given r_ij (R9) */
static double pair_ik_weight(const orc_dpd_params* p, const orc_box* b, int i, const double dr[3]) {
  if (p->flow_mode != ORC_FLOW_AFBC) return 1.0;
  double a[3], c[3], half[3];
  rel_pos(b, i, a);
  for (int k = 0; k < 3; ++k) {
    c[k] = a[k] - dr[k];               /* image of j next to i */
    half[k] = 0.5 * p->core_frac * b->edge[k];
  }
  if (p->dim == 2) half[2] = HUGE_VAL;  /* no z extent in 2D */
  return orc_segment_fraction(a, c, half);
}

static void add_virial(double v6[6], double w, const double F[3], const double dr[3]) {
  v6[0] += w * F[0] * dr[0];
  v6[1] += w * F[1] * dr[1];
  v6[2] += w * F[2] * dr[2];
  v6[3] += w * F[0] * dr[1];
  v6[4] += w * F[0] * dr[2];
  v6[5] += w * F[1] * dr[2];
}

/* Visit every ordered pair (i, j != i): F_i = sum_j F_ij (Eq. F_DPD) plus the
 * FENE terms of i's bonds (Eq. motion).  The virial is half the sum over
 * ordered pairs, i.e. the sum over unordered pairs. */
static int accumulate_pair(const orc_dpd_params* p, orc_box* b, double gdot, int i, int j,
                           double* Fi, double v6[6]) {
  double dr[3], dv[3], F[3];
  int hit, err = 0;
  pair_disp(p, b, gdot, i, j, dr, dv);
  if (!excluded(p, b, i, j)) {
    dpd_pair_force(p, b, i, j, dr, dv, F, &hit);
    if (hit) {
      Fi[0] += F[0]; Fi[1] += F[1]; Fi[2] += F[2];
      add_virial(v6, 0.5 * pair_ik_weight(p, b, i, dr), F, dr);
    }
  }
  (void)err;
  return 0;
}

static int add_bonds(const orc_dpd_params* p, orc_box* b, double gdot, int i, double* Fi,
                     double v6[6]) {
  int err = 0;
  int np = b->n_chains * b->chain_len;
  if (i >= np) return 0;
  int nb[2] = {-1, -1};
  if (i % b->chain_len != 0) nb[0] = i - 1;
  if ((i + 1) % b->chain_len != 0) nb[1] = i + 1;
  for (int k = 0; k < 2; ++k) {
    int j = nb[k];
    if (j < 0) continue;
    double dr[3], dv[3], F[3];
    pair_disp(p, b, gdot, i, j, dr, dv);
    if (fene_force(p, dr, F)) err |= ORC_ERR_BOND_OVERSTRETCH;
    Fi[0] += F[0]; Fi[1] += F[1]; Fi[2] += F[2];
    add_virial(v6, 0.5 * pair_ik_weight(p, b, i, dr), F, dr);
  }
  return err;
}

int orc_compute_forces(const orc_dpd_params* p, orc_box* b, const double L[9], int brute,
                       double virial6[6]) {
  const int n = b->n;
  const double gdot = lees_edwards_rate(p, L);
  int err = 0;
  double v6[6] = {0, 0, 0, 0, 0, 0};
  int nc[3];
  for (int a = 0; a < 3; ++a) {
    nc[a] = (int)floor(b->edge[a] / p->rc);
    if (a == 2 && p->dim == 2) nc[a] = 1; /* one layer, z = 0 */
    else if (nc[a] < 3) return ORC_ERR_ARG;
  }
  const int dz_max = p->dim == 2 ? 0 : 1;
  for (int k = 0; k < 3 * n; ++k) b->force[k] = 0.0;

  if (brute) {
    for (int i = 0; i < n; ++i) {
      double* Fi = &b->force[3 * i];
      for (int j = 0; j < n; ++j)
        if (j != i) accumulate_pair(p, b, gdot, i, j, Fi, v6);
      err |= add_bonds(p, b, gdot, i, Fi, v6);
    }
  } else {
    /* linked cells of width >= rc (Allen & Tildesley) */
    const int ncell = nc[0] * nc[1] * nc[2];
    int* head = (int*)malloc(sizeof(int) * ncell);
    int* next = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    int* cellof = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int c = 0; c < ncell; ++c) head[c] = -1;
    for (int i = 0; i < n; ++i) {
      int ci[3];
      for (int a = 0; a < 3; ++a) {
        ci[a] = (int)floor(b->pos[3 * i + a] / (b->edge[a] / nc[a]));
        if (ci[a] < 0) ci[a] = 0;
        if (ci[a] >= nc[a]) ci[a] = nc[a] - 1;
      }
      int c = ci[0] + nc[0] * (ci[1] + nc[1] * ci[2]);
      cellof[i] = c;
      next[i] = head[c];
      head[c] = i;
    }
    for (int i = 0; i < n; ++i) {
      double* Fi = &b->force[3 * i];
      int c = cellof[i];
      int cx = c % nc[0], cy = (c / nc[0]) % nc[1], cz = c / (nc[0] * nc[1]);
      for (int dz = -dz_max; dz <= dz_max; ++dz) {
        int z = (cz + dz + nc[2]) % nc[2];
        for (int dy = -1; dy <= 1; ++dy) {
          int yraw = cy + dy;
          int y = (yraw + nc[1]) % nc[1];
          int crosses = (yraw < 0 || yraw >= nc[1]);
          /* a row across the sheared y boundary: its images slide in x, so
           * every x cell of that row is a candidate (superset, no duplicates) */
          int xall = (p->flow_mode == ORC_FLOW_LEES_EDWARDS) && crosses;
          int xlo = xall ? 0 : -1, xhi = xall ? nc[0] - 1 : 1;
          for (int dx = xlo; dx <= xhi; ++dx) {
            int x = xall ? dx : (cx + dx + nc[0]) % nc[0];
            int cc = x + nc[0] * (y + nc[1] * z);
            for (int j = head[cc]; j >= 0; j = next[j])
              if (j != i) accumulate_pair(p, b, gdot, i, j, Fi, v6);
          }
        }
      }
      err |= add_bonds(p, b, gdot, i, Fi, v6);
    }
    free(head); free(next); free(cellof);
  }
  for (int k = 0; k < 3 * n; ++k)
    if (!isfinite(b->force[k])) { err |= ORC_ERR_NAN; break; }
  if (virial6) for (int k = 0; k < 6; ++k) virial6[k] = v6[k];
  return err;
}

/* streaming velocity at bead i (R7, R8) */
static void streaming_velocity(const orc_dpd_params* p, const orc_box* b, const double L[9],
                               int i, double u[3]) {
  u[0] = u[1] = u[2] = 0.0;
  if (p->flow_mode == ORC_FLOW_LEES_EDWARDS) {
    u[0] = lees_edwards_rate(p, L) * (b->pos[3 * i + 1] - 0.5 * b->edge[1]);
  } else if (p->flow_mode == ORC_FLOW_AFBC) {
    double rp[3];
    rel_pos(b, i, rp);
    for (int a = 0; a < 3; ++a)
      u[a] = p->lambda_star * (L[3 * a + 0] * rp[0] + L[3 * a + 1] * rp[1] + L[3 * a + 2] * rp[2]);
  }
}

/* Eqs. IKtotal, kinetic_stress, potential_stress for one time sample, with
 * the virial of the current forces supplied (R9). */
static void ik_from_virial(const orc_dpd_params* p, const orc_box* b, const double L[9],
                           const double v6[6], double pi6[6]) {
  double K[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < b->n; ++i) {
    if (p->flow_mode == ORC_FLOW_AFBC && orc_afbc_region(p, b->edge, &b->pos[3 * i]) != 0)
      continue;
    double u[3], dv[3];
    streaming_velocity(p, b, L, i, u);
    for (int a = 0; a < 3; ++a) dv[a] = b->vel[3 * i + a] - u[a];
    K[0] += p->mass * dv[0] * dv[0];
    K[1] += p->mass * dv[1] * dv[1];
    K[2] += p->mass * dv[2] * dv[2];
    K[3] += p->mass * dv[0] * dv[1];
    K[4] += p->mass * dv[0] * dv[2];
    K[5] += p->mass * dv[1] * dv[2];
  }
  double V = core_volume(p, b);
  for (int k = 0; k < 6; ++k) pi6[k] = -(K[k] + v6[k]) / V;
}

int orc_ik_sample(const orc_dpd_params* p, orc_box* b, const double L[9], double pi6[6]) {
  double v6[6];
  double* save = (double*)malloc(sizeof(double) * 3 * (b->n > 0 ? b->n : 1));
  memcpy(save, b->force, sizeof(double) * 3 * b->n);
  int err = orc_compute_forces(p, b, L, 0, v6);
  memcpy(b->force, save, sizeof(double) * 3 * b->n);
  free(save);
  ik_from_virial(p, b, L, v6, pi6);
  return err;
}

/* Conserved quantities of Eq. motion without dissipation: total momentum,
 * kinetic energy and the potentials whose negative gradients are the
 * conservative force (Eq. conservative: a (1 - r/rc) = -d/dr [a rc/2
 * (1 - r/rc)^2]) and the FENE force (Eq. fene_force, R4: -H r/(1 - r^2/R0^2)
 * = -d/dr [-H R0^2/2 ln(1 - r^2/R0^2)]). */
int orc_diagnostics(const orc_dpd_params* p, const orc_box* b, const double L[9], double out[8]) {
  const double gdot = lees_edwards_rate(p, L);
  int err = 0;
  double P[3] = {0, 0, 0}, kin = 0.0, uc = 0.0, uf = 0.0;
  for (int i = 0; i < b->n; ++i) {
    double v2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      P[a] += p->mass * b->vel[3 * i + a];
      v2 += b->vel[3 * i + a] * b->vel[3 * i + a];
    }
    kin += 0.5 * p->mass * v2;
  }
  orc_box* bb = (orc_box*)b; /* pair_disp reads only */
  for (int i = 0; i < b->n; ++i) {
    for (int j = i + 1; j < b->n; ++j) {
      double dr[3], dv[3];
      pair_disp(p, bb, gdot, i, j, dr, dv);
      const double r = sqrt(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
      if (r < p->rc && !excluded(p, bb, i, j)) {
        const double w = 1.0 - r / p->rc;
        uc += 0.5 * p->a_ij * p->rc * w * w;
      }
    }
  }
  const int np = b->n_chains * b->chain_len;
  for (int i = 0; i + 1 < np; ++i) {
    if ((i + 1) % b->chain_len == 0) continue; /* chain end */
    double dr[3], dv[3];
    pair_disp(p, bb, gdot, i, i + 1, dr, dv);
    double x = (dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]) / (p->R0 * p->R0);
    if (!(x < 1.0)) { x = 0.99; err |= ORC_ERR_BOND_OVERSTRETCH; }
    uf += -0.5 * p->H_fene * p->R0 * p->R0 * log(1.0 - x);
  }
  out[0] = P[0]; out[1] = P[1]; out[2] = P[2];
  out[3] = kin; out[4] = uc; out[5] = uf; out[6] = kin + uc + uf; out[7] = 0.0;
  return err;
}

/* velocity-Verlet steps (R6) with the imposed flow (R7, R8) and an IK sample
 * after each full step; time average over the call (Eq. kinetic_stress,
 * N'_t = n_steps) scaled by alpha/lambda* (Eq. pip). */
int orc_advance(const orc_dpd_params* p, orc_box* b, const double L[9], int n_steps,
                double stress_mean[6], double stress_sq[6]) {
  const int n = b->n;
  const double dt = p->dt, hm = 0.5 * p->dt / p->mass;
  const double gdot = lees_edwards_rate(p, L);
  double sum[6] = {0, 0, 0, 0, 0, 0}, sq[6] = {0, 0, 0, 0, 0, 0};
  int err = 0;
  for (int s = 0; s < n_steps; ++s) {
    for (int k = 0; k < 3 * n; ++k) b->vel[k] += hm * b->force[k];
    if (p->flow_mode == ORC_FLOW_LEES_EDWARDS)
      b->le_offset = wrap_to(b->le_offset + gdot * b->edge[1] * dt, b->edge[0]);
    for (int i = 0; i < n; ++i) {
      double* r = &b->pos[3 * i];
      double* v = &b->vel[3 * i];
      for (int a = 0; a < 3; ++a) r[a] += dt * v[a];
      if (p->flow_mode == ORC_FLOW_LEES_EDWARDS) {
        if (r[1] >= b->edge[1]) { r[1] -= b->edge[1]; r[0] -= b->le_offset; v[0] -= gdot * b->edge[1]; }
        else if (r[1] < 0.0) { r[1] += b->edge[1]; r[0] += b->le_offset; v[0] += gdot * b->edge[1]; }
      }
      for (int a = 0; a < 3; ++a) r[a] = wrap_to(r[a], b->edge[a]);
    }
    b->step += 1;
    double v6[6];
    err |= orc_compute_forces(p, b, L, 0, v6);
    for (int k = 0; k < 3 * n; ++k) b->vel[k] += hm * b->force[k];
    if (p->flow_mode == ORC_FLOW_AFBC && p->afbc_mode == 1) {
      /* R8 alternative: BC beads keep their velocity about the mean of the BC
       * beads of their cell; cells are the linked cells of the pair search,
       * n_c = floor(E / rc) per axis of width exactly E / n_c. */
      int nc[3];
      double wf[3];
      for (int a = 0; a < 3; ++a) {
        nc[a] = (a == 2 && p->dim == 2) ? 1 : (int)floor(b->edge[a] / p->rc);
        wf[a] = b->edge[a] / (double)nc[a];
      }
      const int ncell = nc[0] * nc[1] * nc[2];
      double* sum = (double*)calloc((size_t)ncell * 4, sizeof(double));
      int* cell = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
      for (int i = 0; i < n; ++i) {
        int ci[3];
        for (int a = 0; a < 3; ++a) {
          ci[a] = (int)floor(b->pos[3 * i + a] / wf[a]);
          if (ci[a] < 0) ci[a] = 0;
          if (ci[a] >= nc[a]) ci[a] = nc[a] - 1;
        }
        cell[i] = ci[0] + nc[0] * (ci[1] + nc[1] * ci[2]);
        if (orc_afbc_region(p, b->edge, &b->pos[3 * i]) != 1) continue;
        for (int a = 0; a < 3; ++a) sum[4 * cell[i] + a] += b->vel[3 * i + a];
        sum[4 * cell[i] + 3] += 1.0;
      }
      for (int i = 0; i < n; ++i) {
        if (orc_afbc_region(p, b->edge, &b->pos[3 * i]) != 1) continue;
        double u[3];
        streaming_velocity(p, b, L, i, u);
        const double* m = &sum[4 * cell[i]];
        for (int a = 0; a < 3; ++a) b->vel[3 * i + a] = u[a] + (b->vel[3 * i + a] - m[a] / m[3]);
      }
      free(sum);
      free(cell);
    } else if (p->flow_mode == ORC_FLOW_AFBC) {
      for (int i = 0; i < n; ++i) {
        if (orc_afbc_region(p, b->edge, &b->pos[3 * i]) != 1) continue;
        double u[3];
        streaming_velocity(p, b, L, i, u);
        for (int a = 0; a < 3; ++a) b->vel[3 * i + a] = u[a];
      }
    }
    double pi6[6];
    ik_from_virial(p, b, L, v6, pi6);
    for (int k = 0; k < 6; ++k) { sum[k] += pi6[k]; sq[k] += pi6[k] * pi6[k]; }
    if (err & (ORC_ERR_NAN | ORC_ERR_ARG)) break;
  }
  const double scale = p->alpha / p->lambda_star;
  for (int k = 0; k < 6; ++k) {
    double m = n_steps > 0 ? sum[k] / n_steps : 0.0;
    double q = n_steps > 0 ? sq[k] / n_steps : 0.0;
    if (stress_mean) stress_mean[k] = scale * m;
    if (stress_sq) stress_sq[k] = scale * scale * q;
  }
  return err;
}

int orc_advance_batch(const orc_dpd_params* p, orc_box* boxes, int n_boxes, const double* L,
                      int n_steps, double* stress_mean, double* stress_sq, int n_threads,
                      int* status) {
  int err = 0;
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(| : err)
#endif
  for (int k = 0; k < n_boxes; ++k) {
    int e = orc_advance(p, &boxes[k], &L[9 * k], n_steps,
                        stress_mean ? &stress_mean[6 * k] : NULL,
                        stress_sq ? &stress_sq[6 * k] : NULL);
    if (status) status[k] = e;
    err |= e;
  }
  (void)n_threads;
  return err;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
