/*
 * lhmm_oracle.h -- plain, slow, FP64 CPU oracle for the LHMM micro (DPD/FENE)
 * and macro (SPH) hot path of arXiv 2512.13267.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Every function follows the paper's definitions step by step:
 *   DPD equation of motion (Eq. motion), pair forces (Eqs. conservative,
 *   dissipative, random), FDT, FENE spring (Eq. fene_force), velocity-Verlet
 *   (coupling protocol, Step 3), AFBC velocity imposition (Eq. micro_bc),
 *   Irving-Kirkwood stress (Eqs. IKtotal, kinetic_stress, potential_stress),
 *   characteristic-stress scaling (Eq. pip); SPH momentum (Eq.
 *   sph_continuity), Tait EOS (Eq. tait), SPH velocity gradient
 *   (Eq. macro_micro), Lucy kernel (Appendix A).
 * Readings where the paper is silent or garbled are stated at the top of
 * each source file and at the function that uses them.
 */
#ifndef LHMM_ORACLE_H
#define LHMM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_FLOW_PERIODIC = 0, ORC_FLOW_LEES_EDWARDS = 1, ORC_FLOW_AFBC = 2 };

/* error bits returned by the stepping functions */
enum {
  ORC_OK = 0,
  ORC_ERR_BOND_OVERSTRETCH = 1, /* a FENE bond reached |r| >= R0 */
  ORC_ERR_NAN = 2,              /* a non-finite force or velocity */
  ORC_ERR_ARG = 4               /* bad sizes (box smaller than 3 r_c, ...) */
};

typedef struct {
  double a_ij;      /* conservative amplitude (Eq. conservative) */
  double gamma;     /* dissipative coefficient gamma^D (Eq. dissipative) */
  double sigma;     /* random amplitude sigma^R (Eq. random); FDT: sqrt(2 gamma kBT) */
  double kBT;
  double rc;        /* cutoff radius */
  double H_fene;    /* FENE spring constant (Eq. fene_force) */
  double R0;        /* FENE maximum extension */
  double dt;        /* DPD time step */
  double mass;      /* bead mass */
  uint64_t seed;    /* Philox key material */
  int flow_mode;    /* ORC_FLOW_* */
  double core_frac; /* AFBC core width / box width (Table 2: 24/76) */
  double bc_frac;   /* AFBC BC-shell width / box width, each side (Table 2: 13/76) */
  int dpd_on_bonded;/* 1: DPD pair forces also act between bonded beads (sum over all j != i) */
  double alpha;       /* viscosity ratio (Eq. ratios) */
  double lambda_star; /* time-scale ratio (Eq. ratios) */
  int dim;            /* 3, or 2: beads move in the x-y plane (z = 0, z edge unused,
                         one cell layer, no z neighbours); volumes become areas */
  int exclude_bonds;  /* K in 0..3: no DPD pair force between beads of one chain at
                         most K bonds apart (dpd_on_bonded = 0 means at least 1) */
  int afbc_mode;      /* 0: BC beads take v = L r' (R8); 1: they keep their peculiar
                         velocity about the mean of the BC beads of their cell,
                         v = L r' + (v - mean_cell(v)) (R8's alternative) */
} orc_dpd_params;

typedef struct {
  int box_id;        /* index of the box in its batch; part of the Philox key */
  double edge[3];    /* box edges; positions live in [0, edge) */
  int n;             /* beads */
  int n_chains;      /* chains occupy ids [c*chain_len, (c+1)*chain_len) */
  int chain_len;
  double* pos;       /* n x 3 */
  double* vel;       /* n x 3 */
  double* force;     /* n x 3: forces of the current state (F at step `step`) */
  uint64_t step;     /* number of completed steps; keys the random force */
  double le_offset;  /* Lees-Edwards image offset in x, in [0, edge[0]) */
} orc_box;

/* ---------------- random numbers ---------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_pair_theta(uint64_t seed, int box_id, int id_i, int id_j, uint64_t step);
double orc_theta_from_words(uint32_t x0, uint32_t x1);

/* ---------------- micro (DPD / FENE) ---------------- */
/* forces of the current state; virial6 = sum over pairs of B_ij r_ij (x) F_ij
 * (xx, yy, zz, xy, xz, yz), B the IK bond function times V_core.
 * brute = 1 uses an O(N^2) pair search instead of the cell list. */
int orc_compute_forces(const orc_dpd_params* p, orc_box* b, const double L[9],
                       int brute, double virial6[6]);
/* n_steps velocity-Verlet steps; stress_mean/stress_sq = (alpha/lambda*) times
 * the time average of pi_n and of pi_n^2 over the n_steps samples. */
int orc_advance(const orc_dpd_params* p, orc_box* b, const double L[9], int n_steps,
                double stress_mean[6], double stress_sq[6]);
/* the same over many boxes, OpenMP over boxes (n_threads <= 0: all) */
int orc_advance_batch(const orc_dpd_params* p, orc_box* boxes, int n_boxes,
                      const double* L /* n_boxes x 9 */, int n_steps,
                      double* stress_mean /* n_boxes x 6 */, double* stress_sq,
                      int n_threads, int* status /* n_boxes */);
/* one IK sample (no time average, no alpha scaling) from the current state */
int orc_ik_sample(const orc_dpd_params* p, orc_box* b, const double L[9], double pi6[6]);

/* Momentum and energy of one box (Eq. motion's conserved quantities): out =
 * [P_x, P_y, P_z, kinetic sum m v^2 / 2, conservative DPD potential (every
 * non-excluded pair once, U = a rc/2 (1 - r/rc)^2 for r < rc), FENE potential
 * (every bond, U = -H R0^2/2 ln(1 - r^2/R0^2)), total of the three energies,
 * 0].  Brute force over all pairs, minimum images as the forces take them.
 * Returns ORC_ERR_BOND_OVERSTRETCH for a bond at |r| >= R0 (its energy is
 * then taken at (r/R0)^2 = 0.99, reading R10). */
int orc_diagnostics(const orc_dpd_params* p, const orc_box* b, const double L[9], double out[8]);
/* AFBC region of a position: 0 core, 1 BC shell, 2 buffer */
int orc_afbc_region(const orc_dpd_params* p, const double edge[3], const double r[3]);
/* length fraction of the segment a->b inside the centred box |x_k| < half[k] */
double orc_segment_fraction(const double a[3], const double b[3], const double half[3]);
int orc_max_threads(void);

/* ---------------- macro (SPH, 2D) ---------------- */
enum { ORC_KERNEL_WENDLAND_C2 = 0, ORC_KERNEL_LUCY = 1 };
enum { ORC_VISC_DERIVED_2D = 0, ORC_VISC_PAPER_LITERAL = 1 };
enum { ORC_BODY_UNIFORM = 0, ORC_BODY_REVERSE_POISEUILLE = 1 };

typedef struct {
  int n;            /* all particles, walls included */
  double Lx, Ly;    /* periodic box */
  double h;         /* kernel support radius */
  double mass, rho0, c, theta_pb;
  double eta_s, zeta_s;
  double dt;
  int kernel;       /* ORC_KERNEL_* */
  int visc_coeffs;  /* ORC_VISC_* */
  double body_force[2];
  int body_mode;    /* ORC_BODY_* */
} orc_sph_params;

double orc_sph_W(int kernel, double r, double h);
double orc_sph_F(int kernel, double r, double h); /* -W'(r)/r */
double orc_sph_pressure(const orc_sph_params* p, double rho);
/* number densities d_I = sum_J W_IJ (self included) */
void orc_sph_density(const orc_sph_params* p, const double* pos, double* d);
/* accelerations dv/dt of all particles; stress3 = n x 3 (xx, xy, yy) polymer
 * stress already scaled by alpha/lambda* (or NULL). Walls get zero. */
void orc_sph_accel(const orc_sph_params* p, const double* pos, const double* vel,
                   const int* is_wall, const double* stress3, double* acc, double* d_out);
/* velocity gradient L_ab = dv_a/dx_b = sum_J (F_IJ/d_J) v_IJ,a r_IJ,b */
void orc_sph_velgrad(const orc_sph_params* p, const double* pos, const double* vel,
                     const double* d, double* L4 /* n x 4: xx, xy, yx, yy */);
/* n_sub velocity-Verlet steps; acc holds a(t) on entry and a(t+n_sub dt) on exit */
void orc_sph_steps(const orc_sph_params* p, double* pos, double* vel, double* acc,
                   const int* is_wall, const double* stress3, int n_sub);

/* ---------------- learned closure (MLP) ---------------- */
/* dims[0..n_layers]: widths; W_l is dims[l+1] x dims[l] row-major, b_l dims[l+1];
 * GELU (erf form) after every layer but the last.  params holds W_0,b_0,W_1,b_1,...
 * acts (optional) receives every pre-activation and activation for backward. */
long orc_mlp_n_params(int n_layers, const int* dims);
void orc_mlp_forward(int n_layers, const int* dims, const double* params, int batch,
                     const double* x, double* y);
/* loss = mean over batch and outputs of (y - target)^2; grad = d loss / d params */
double orc_mlp_loss_grad(int n_layers, const int* dims, const double* params, int batch,
                         const double* x, const double* target, double* grad);
/* one AdamW step (Loshchilov & Hutter), step count t >= 1 */
void orc_adamw_step(long n, double* params, const double* grad, double* m, double* v,
                    double lr, double beta1, double beta2, double eps, double wd, long t);
double orc_gelu(double x);

#ifdef __cplusplus
}
#endif
#endif
