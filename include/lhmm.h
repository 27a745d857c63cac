/*
 * lhmm.h -- C ABI of the GB300 (sm_103a) LHMM hot path.
 *
 * The Lagrangian Heterogeneous Multiscale Method of arXiv 2512.13267 couples
 * a macroscale SPH fluid to one microscale DPD/FENE polymer box per SPH
 * particle.  Every macro step the SPH velocity gradient goes down to the
 * boxes (Sec. 3.4, Eqs. macro_micro and micro_bc), each box advances k'
 * DPD steps (Sec. 2.3, Eqs. motion..fene_force, coupling protocol Step 3)
 * and returns its time-averaged Irving-Kirkwood polymer stress (Sec. 3.5,
 * Eqs. IKtotal..potential_stress), scaled by alpha/lambda* (Eq. pip), to the
 * SPH momentum equation (Eq. sph_continuity).
 *
 * Conventions shared by every entry point:
 *  - Pointers named *_dev are device pointers, *_host are host pointers.  The
 *    caller owns them; the library never frees or retains them after the call.
 *  - The library owns the handles and all of their internal device state.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls that take a stream only enqueue work and return; calls
 *    documented as synchronous wait for their own work.
 *  - Arguments are checked on the host; a bad argument returns LHMM_ERR_ARG
 *    and enqueues nothing.  No call aborts, traps or prints.
 *  - Errors detected on the device (bond over-stretch, NaN) are kept in a
 *    per-box status word and reported by lhmm_micro_sync.
 *  - Handles are not thread-safe: one host thread per handle at a time.
 *  - Tensor layouts: a velocity gradient L is 9 floats, row-major,
 *    L[3a+b] = du_a/dx_b (so the imposed streaming velocity is u = L r).  A
 *    stress is 6 doubles in the order xx, yy, zz, xy, xz, yz.
 */
#ifndef LHMM_H
#define LHMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LHMM_OK = 0,
  LHMM_ERR_ARG = 1,             /* invalid argument, nothing enqueued */
  LHMM_ERR_CUDA = 2,            /* a CUDA runtime call failed */
  LHMM_ERR_OOM = 3,             /* device allocation failed */
  LHMM_ERR_BOND_OVERSTRETCH = 4,/* a FENE bond reached |r| >= R0 (Eq. fene_force undefined) */
  LHMM_ERR_CELL_OVERFLOW = 5,   /* a box outgrew its shared-memory plan */
  LHMM_ERR_NAN = 6,             /* a non-finite bead velocity or force */
  LHMM_ERR_TIMEOUT = 7,         /* a bounded device wait gave up */
  LHMM_ERR_UNSUPPORTED = 8,     /* a configuration this build does not run */
  LHMM_ERR_FORCE_RANGE = 9      /* a pair force component exceeded 512 (clamped) */
} lhmm_status;

/* per-box device status bits, as returned by lhmm_micro_sync */
#define LHMM_BOX_BOND_OVERSTRETCH 1u
#define LHMM_BOX_NAN 2u
#define LHMM_BOX_CELL_OVERFLOW 4u
#define LHMM_BOX_FORCE_RANGE 8u

/* imposed-flow treatment of the micro boxes */
#define LHMM_FLOW_PERIODIC 0     /* plain periodic box, no imposed flow */
#define LHMM_FLOW_LEES_EDWARDS 1 /* sliding-brick images for shear du_x/dy = L[1] */
#define LHMM_FLOW_AFBC 2         /* arbitrary-flow boundary conditions (Sec. 4.1, Table 2) */

/* DPD/FENE parameters (Sec. 2.3; Table 1 for the paper's melts).
 * sigma should satisfy the FDT sigma^2 = 2 gamma kBT; it is not enforced. */
typedef struct {
  float a_ij;        /* conservative amplitude, Eq. conservative */
  float gamma;       /* dissipative coefficient gamma^D, Eq. dissipative */
  float sigma;       /* random amplitude sigma^R, Eq. random */
  float kBT;         /* thermal energy (used for documentation/diagnostics) */
  float rc;          /* cutoff radius; cells are >= rc wide */
  float H_fene;      /* FENE spring constant, Eq. fene_force */
  float R0;          /* FENE maximum bond extension */
  float dt;          /* DPD time step */
  float mass;        /* bead mass */
  uint64_t seed;     /* key of the counter-based random stream */
  int flow_mode;     /* LHMM_FLOW_* */
  float afbc_core_frac; /* AFBC core width / box edge (Table 2: 24/76) */
  float afbc_bc_frac;   /* AFBC BC shell width / box edge, per side (Table 2: 13/76) */
  int dpd_on_bonded;    /* 1: DPD pair forces also act on bonded pairs (sum over all j != i) */
  double alpha;         /* viscosity ratio alpha, Eq. ratios; output is scaled by alpha/lambda* */
  double lambda_star;   /* time-scale ratio lambda*, Eq. ratios; input L is scaled by lambda* */
  int dim;              /* 3, or 2 for the paper's planar melt boxes (Table 1): beads move in
                           the x-y plane (z components of positions, velocities and forces are
                           set to 0, the z edge is ignored), one cell layer, pairs in the plane,
                           AFBC squares, IK stress per core area.  0 means 3; other values
                           return LHMM_ERR_ARG. */
  int exclude_bonds;    /* K in 0..3: no DPD pair force (C, D, R) between beads of one chain
                           at most K bonds apart (LAMMPS special_bonds lj 0 0 0 is K = 3);
                           dpd_on_bonded = 0 means K >= 1.  FENE bonds are unaffected.
                           Other values return LHMM_ERR_ARG. */
  int afbc_mode;        /* 0: every BC-shell bead takes v = lambda* L r' after the second
                           half kick (Eq. micro_bc, full overwrite); 1: it keeps its
                           velocity about the mean of the BC beads of its cell,
                           v = lambda* L r' + (v - mean_cell(v)), so the shell stays
                           thermal.  Other values return LHMM_ERR_ARG. */
} lhmm_dpd_params;

/* A batch of independent boxes.  Box b has edges box_edge[3b..3b+2] (its
 * beads live in [0, edge)), n_beads[b] beads with ids 0..n_beads[b]-1, and
 * n_chains[b] FENE chains of chain_len consecutive ids starting at id 0
 * (bonds (k, k+1) inside a chain); the remaining ids are solvent.  Beads of
 * all boxes are concatenated in box order in every per-bead array. */
typedef struct {
  int n_boxes;
  const float* box_edge; /* host, n_boxes x 3; every edge >= 3 rc */
  const int* n_beads;    /* host, n_boxes; 0 <= n < 65536 */
  const int* n_chains;   /* host, n_boxes; n_chains * chain_len <= n_beads */
  int chain_len;         /* N_d >= 2 (ignored when every n_chains is 0) */
  int box_id_offset;     /* >= 0: box b of this batch keys its random stream as box
                            box_id_offset + b, so a batch that holds boxes lo..hi-1 of a
                            larger system (one rank's share) draws the same noise as
                            those boxes do in one batch of the whole system; 0 otherwise */
} lhmm_batch_desc;

typedef struct lhmm_micro_s* lhmm_micro_t;

const char* lhmm_status_string(lhmm_status s);

/* Create a batch of micro-domains from initial bead states (host,
 * total_beads x 3: absolute positions inside each box as double, velocities
 * as float), and
 * compute the initial forces F(0) under the velocity gradients L0_host (host,
 * n_boxes x 9, or NULL for zero; Lees-Edwards boxes need it for the velocity
 * jump of their sliding images).  Synchronous.  Allocates all device state,
 * including the per-box scratch of the device-memory kernel variants when
 * the largest box does not fit one SM's shared memory.  Returns
 * LHMM_ERR_ARG for bad sizes or parameters, LHMM_ERR_UNSUPPORTED for a box
 * of more than 65 535 cells or a Lees-Edwards box of more than 60 cells in
 * x (16-bit cell ids and the 8-bit image offset of a queued pair). */
lhmm_status lhmm_micro_create(const lhmm_dpd_params* params, const lhmm_batch_desc* batch,
                              const double* pos0_host, const float* vel0_host,
                              const float* L0_host, void* stream, lhmm_micro_t* out);
lhmm_status lhmm_micro_destroy(lhmm_micro_t h);

/* Advance boxes by n_steps velocity-Verlet DPD steps (coupling protocol,
 * Step 3) under their velocity gradients, and write the time average over
 * those steps of the IK stress (Eqs. IKtotal..potential_stress, sampled after
 * each full step) times alpha/lambda* (Eq. pip).
 *   L_dev         device, n_boxes x 9 float, indexed by box id; scaled by
 *                 lambda* inside (Eq. micro_bc).  PERIODIC ignores it,
 *                 LEES_EDWARDS reads only L[1] = du_x/dy.
 *   box_idx_dev   device, n_active box ids to advance, or NULL for all boxes
 *                 (then n_active must equal n_boxes); ids must be distinct.
 *   n_steps       >= 0 (k' of the coupling interval)
 *   stress_dev    device, n_boxes x 6 double, rows indexed by box id; only
 *                 the advanced boxes' rows are written.
 *   stress_sq_dev device, n_boxes x 6 double or NULL: time average of the
 *                 square of each per-step sample (for standard errors).
 * Asynchronous on `stream`.  Device-side errors surface in lhmm_micro_sync. */
lhmm_status lhmm_micro_advance(lhmm_micro_t h, const float* L_dev, const int* box_idx_dev,
                               int n_active, int n_steps, double* stress_dev,
                               double* stress_sq_dev, void* stream);

/* The same over a box list whose length is known only on the device (e.g. the
 * output of a gate): the boxes box_idx_dev[0 .. min(*n_active_dev, max_active))
 * are advanced by a persistent launch whose blocks take list items from a
 * device counter.  max_active <= n_boxes bounds the list.  Asynchronous;
 * capturable in a CUDA graph. */
lhmm_status lhmm_micro_advance_dev_count(lhmm_micro_t h, const float* L_dev,
                                         const int* box_idx_dev, const int* n_active_dev,
                                         int max_active, int n_steps, double* stress_dev,
                                         double* stress_sq_dev, void* stream);

/* FP64 momentum and energy of every box of the current state (Eq. motion:
 * without its dissipative and random terms the dynamics conserve the total
 * momentum and the energy below; with them the momentum is still conserved).
 *   diag_dev  device, n_boxes x 8 double, row b = [P_x, P_y, P_z,
 *             kinetic energy sum m v^2/2, conservative DPD potential
 *             sum over non-excluded pairs within rc of a rc/2 (1 - r/rc)^2
 *             (the potential of Eq. conservative), FENE potential sum over
 *             bonds of -H R0^2/2 ln(1 - r^2/R0^2) (Eq. fene_force),
 *             total energy (the sum of the three), 1 if a bond was at
 *             |r| >= R0 (its energy then taken at (r/R0)^2 = 0.99) else 0].
 * Sums are accumulated in FP64 from the FP32 state; pairs by brute force
 * over each box with minimum images (Lees-Edwards shifted across y), so the
 * cost is O(N^2) per box: a diagnostic, not a per-step call.  Velocities are
 * lab-frame (the imposed flow is not subtracted).  Asynchronous on `stream`;
 * reads the state the last advance left. */
lhmm_status lhmm_micro_diagnostics(lhmm_micro_t h, double* diag_dev, void* stream);

/* The same over host buffers: copies L_host (n_boxes x 9) in, advances all
 * boxes, copies stress (n_boxes x 6) and optionally stress_sq back, and waits
 * for the stream.  Synchronous.  Uses staging buffers owned by the handle. */
lhmm_status lhmm_micro_advance_host(lhmm_micro_t h, const float* L_host, int n_steps,
                                    double* stress_host, double* stress_sq_host, void* stream);

/* Wait for the handle's stream work, read the per-box status words into
 * box_status_host (n_boxes uint32, or NULL), clear them, and return the first
 * error they hold (LHMM_ERR_BOND_OVERSTRETCH, LHMM_ERR_NAN,
 * LHMM_ERR_CELL_OVERFLOW, LHMM_ERR_FORCE_RANGE) or LHMM_OK.  Synchronous. */
lhmm_status lhmm_micro_sync(lhmm_micro_t h, uint32_t* box_status_host);

/* Copy one box's state to the host: absolute positions (n x 3 double; the
 * library keeps FP32 offsets inside cells, and a double holds cell origin plus
 * offset exactly), velocities and the forces of the current state (the ones
 * the next half kick uses), its completed step count and Lees-Edwards offset.
 * Any pointer may be NULL.  Synchronous. */
lhmm_status lhmm_micro_get_state(lhmm_micro_t h, int box, double* pos_host, float* vel_host,
                                 float* force_host, uint64_t* step, float* le_offset);
/* Overwrite one box's state (checkpoint/resume).  pos/vel/force are required;
 * the random stream continues from `step`, so a state saved with get_state
 * resumes bit for bit.  Synchronous. */
lhmm_status lhmm_micro_set_state(lhmm_micro_t h, int box, const double* pos_host,
                                 const float* vel_host, const float* force_host, uint64_t step,
                                 float le_offset);

/* Sizes of the batch. */
lhmm_status lhmm_micro_info(lhmm_micro_t h, int* n_boxes, int64_t* total_beads, int* max_beads);

/* Launch plan (not in the paper; the batching layer of this library).  Boxes
 * are grouped into size classes of similar bead count; each class runs as one
 * launch on a stream of its own (forked from and joined back into the caller's
 * stream), with a shared-memory plan sized to its largest box and one of
 * LHMM_MICRO_N_VARIANTS kernel variants (threads per block x resident blocks
 * per SM).  A subset advance (box_idx_dev != NULL) is one launch sized to the
 * largest box of the batch.
 * Variants 0..4 hold a box in one SM's shared memory (up to about 5 700
 * beads in 3D).  Variants 5 (512 threads) and 6 (256 threads x 2 blocks) hold
 * it in a per-box scratch buffer in device memory, served by L1/L2, for boxes
 * beyond that (up to 65 535 beads and 65 535 cells; the paper's 76 x 76 melt
 * box has 23 104); the handle allocates that buffer (n_boxes x the largest
 * box's plan) when a class needs it or a class is pinned to such a variant.
 * Both kinds run the same arithmetic in the same order, so they give
 * bit-identical results. */
#define LHMM_MICRO_N_VARIANTS 7

/* Time every variant on probe_steps steps of each class's boxes under L_dev
 * (device, n_boxes x 9) and keep the fastest per class; results are cached
 * per (largest box, cells, flow mode, device) for the process.  Then the
 * tuned class plan is timed against one persistent launch over every box
 * (a grid of resident blocks pulling box ids, largest box first, from a
 * device counter) in each variant that holds the largest box, and full
 * advances (box_idx_dev == NULL) use the faster (lhmm_micro_plan then reports
 * the persistent launch as one class).  The bead state
 * is saved before and restored after, so the batch does not advance.  The
 * choice changes floating-point summation order, so a run is bit-reproducible
 * for a fixed plan (see lhmm_micro_set_variant).  Synchronous; allocates a
 * temporary copy of the bead state. */
lhmm_status lhmm_micro_autotune(lhmm_micro_t h, const float* L_dev, int probe_steps, void* stream);

/* Read the plan: the number of classes, and for the first `cap` classes their
 * box count, largest box, threads per block and resident blocks per SM. */
lhmm_status lhmm_micro_plan(lhmm_micro_t h, int* n_classes, int cap, int* class_boxes,
                            int* class_max_beads, int* class_threads, int* class_min_blocks);

/* Pin the kernel variant (0..LHMM_MICRO_N_VARIANTS-1) of one class (this
 * returns full advances to the class plan).  Returns
 * LHMM_ERR_UNSUPPORTED if that variant's shared-memory plan does not fit.
 * Pinning a device-memory variant (5, 6) may allocate the scratch buffer:
 * call it before capturing advances into a CUDA graph. */
lhmm_status lhmm_micro_set_variant(lhmm_micro_t h, int cls, int variant);

/* Pin the kernel variant of the launches over a box list (advances with
 * box_idx_dev, lhmm_micro_advance_dev_count and so the DPD boxes of a gated
 * coupled step); -1 restores the default, which picks the shape by the
 * number of listed boxes: up to one box per SM, one block per SM with as
 * many threads as the largest box's shared-memory plan allows (1024, else
 * 512), so that each box finishes in the fewest clocks; more boxes, two
 * blocks of 512 threads per SM where the box fits that plan.  Boxes no
 * shared-memory plan holds use the device-memory variant 5.  For
 * lhmm_micro_advance_dev_count the count is on the device, so both launches
 * are queued and each leaves the boxes to the other outside its range.  Returns LHMM_ERR_UNSUPPORTED if the variant does
 * not hold the largest box.  Results equal a full advance's bit for bit in
 * positions and velocities; the stress averages equal them to FP32
 * summation order, and bit for bit when both use the same variant.  Call it
 * before capturing advances into a CUDA graph. */
lhmm_status lhmm_micro_set_list_variant(lhmm_micro_t h, int variant);

/* ------------------------------------------------------------------------
 * Macroscale SPH (Sec. 3.2, Eqs. sph_continuity and tait; Sec. 3.4,
 * Eq. macro_micro).  2D periodic box [0,Lx) x [0,Ly); particles 0..n-n_wall-1
 * are fluid and carry micro-domain (box) I = particle I; the last n_wall
 * particles are fixed wall particles (v = 0) that take part in the density,
 * pressure and viscous sums and carry no micro stress.
 * ------------------------------------------------------------------------ */
#define LHMM_SPH_WENDLAND_C2 0       /* W = 7/(pi h^2) (1+4q)(1-q)^4, support h */
#define LHMM_SPH_LUCY 1              /* W = 5/(pi h^2) (1+3q)(1-q)^3 (Appendix A) */
#define LHMM_SPH_VISC_DERIVED_2D 0   /* a = 2 eta - zeta, b = 4 zeta: shear viscosity eta in 2D */
#define LHMM_SPH_VISC_PAPER_LITERAL 1/* a = 2 eta - zeta, b = 4 zeta + 2 eta as printed */
#define LHMM_SPH_BODY_UNIFORM 0      /* body acceleration body_force everywhere */
#define LHMM_SPH_BODY_REVERSE_POISEUILLE 1 /* +F_x for y >= Ly/2, -F_x below (Sec. 6.1) */

typedef struct {
  int n;            /* particles, walls included */
  int n_wall;       /* the last n_wall particles are walls */
  float Lx, Ly;     /* periodic box, each >= 2 h */
  float h;          /* kernel support radius */
  float mass;       /* particle mass m_I */
  float rho0;       /* reference density of the Tait EOS */
  float c;          /* artificial sound speed */
  float theta_pb;   /* background pressure p_b = theta c^2 rho0 / 7 */
  float eta_s;      /* solvent shear viscosity */
  float zeta_s;     /* solvent bulk viscosity */
  float dt;         /* SPH time step */
  int kernel;       /* LHMM_SPH_WENDLAND_C2 | LHMM_SPH_LUCY */
  int visc_coeffs;  /* LHMM_SPH_VISC_* */
  float body_force[2]; /* body acceleration (x, y); F = body_force[0] for RPF */
  int body_mode;    /* LHMM_SPH_BODY_* */
} lhmm_sph_params;

typedef struct lhmm_sph_s* lhmm_sph_t;

/* Create from initial positions and velocities (host, n x 2 float; wall
 * velocities are ignored) and compute the initial accelerations with zero
 * micro stress.  Synchronous; allocates the particle state and its cell list. */
lhmm_status lhmm_sph_create(const lhmm_sph_params* params, const float* pos0_host,
                            const float* vel0_host, void* stream, lhmm_sph_t* out);
lhmm_status lhmm_sph_destroy(lhmm_sph_t h);

/* n_substeps velocity-Verlet SPH steps (coupling protocol Step 1) with the
 * polymer stress held fixed, then, if L_out_dev != NULL, the velocity
 * gradient of every fluid particle (Step 2).
 *   stress_dev  device, (n - n_wall) x 6 double in the layout lhmm_micro_advance
 *               writes (xx, yy, zz, xy, xz, yz; already scaled by alpha/lambda*),
 *               or NULL for no micro stress.  Only xx, xy, yy enter the 2D sum.
 *   L_out_dev   device, (n - n_wall) x 9 float, row-major L_ab = dv_a/dx_b with
 *               the z row and column zero: the input lhmm_micro_advance takes.
 * The first half kick uses the accelerations of the last force evaluation.
 * Asynchronous on `stream`. */
lhmm_status lhmm_sph_step(lhmm_sph_t h, const double* stress_dev, int n_substeps,
                          float* L_out_dev, void* stream);

/* Re-evaluate density, pressure and accelerations at the current state with
 * the given stress (e.g. right after a new micro stress arrives).  Async. */
lhmm_status lhmm_sph_recompute_forces(lhmm_sph_t h, const double* stress_dev, void* stream);

/* Copy positions, velocities, accelerations (n x 2 float) and number
 * densities (n float) to the host; any pointer may be NULL.  Synchronous. */
lhmm_status lhmm_sph_get_state(lhmm_sph_t h, float* pos_host, float* vel_host, float* acc_host,
                               float* density_host);

/* Particle counts of an SPH handle. */
lhmm_status lhmm_sph_info(lhmm_sph_t h, int* n, int* n_wall);

/* ------------------------------------------------------------------------
 * The coupled macro step (coupling protocol, Steps 1-4; time coupling
 * delta_t = M dt_SPH = k' dt_DPD, Eq. in Sec. 3.3.1).  Ties one SPH handle to
 * one micro handle with a box per fluid particle (box I <-> particle I).  One
 * macro step: lhmm_sph_step with the current polymer stress and M substeps,
 * writing the velocity gradients; then lhmm_micro_advance of every box by k'
 * steps under them, writing the new stress.  The two exchange buffers are
 * device arrays owned by the coupled handle.  The caller keeps ownership of
 * the SPH and micro handles and must keep them alive.
 * ------------------------------------------------------------------------ */
typedef struct lhmm_coupled_s* lhmm_coupled_t;

lhmm_status lhmm_coupled_create(lhmm_sph_t sph, lhmm_micro_t micro, int sph_substeps,
                                int micro_steps, lhmm_coupled_t* out);
lhmm_status lhmm_coupled_destroy(lhmm_coupled_t c);

/* Enqueue n_macro macro steps on `stream`.  With use_graph != 0 the first step
 * runs eagerly, the second captures one macro step into a CUDA graph, and
 * every later step replays it (launch overhead of the ~2M+10 kernels of a
 * step collapses to one graph launch).  Asynchronous. */
lhmm_status lhmm_coupled_step(lhmm_coupled_t c, int n_macro, int use_graph, void* stream);

/* Device pointers of the exchange buffers: velocity gradients (n_boxes x 9
 * float) and polymer stresses (n_boxes x 6 double). */
lhmm_status lhmm_coupled_exchange(lhmm_coupled_t c, float** L_dev, double** stress_dev);

/* Wait for the device and copy the exchange buffers to the host (either
 * pointer may be NULL).  Synchronous. */
lhmm_status lhmm_coupled_copy_exchange(lhmm_coupled_t c, float* L_host, double* stress_host);

/* ------------------------------------------------------------------------
 * Learned stress closure (not in the paper; the surrogate layer of this
 * library).  An ensemble of `members` MLPs in -> hidden x n_hidden -> out with
 * exact GELU after every hidden layer, BF16 weights on the tensor cores with
 * FP32 accumulation and FP32 master weights, trained with AdamW (Loshchilov &
 * Hutter) by this library's own forward and backward kernels.  Inputs are
 * normalised per feature ((x - mean)/std) and targets scaled per output by
 * out_scale (lhmm_closure_set_normalization); predictions come back in the
 * target's units.
 * ------------------------------------------------------------------------ */
typedef struct lhmm_closure_s* lhmm_closure_t;

/* members 1..16, hidden a multiple of 32, n_hidden 1..6, out_dim 1..8; weights
 * He-initialised from `seed`, biases zero.  Synchronous; allocates. */
lhmm_status lhmm_closure_create(int members, int in_dim, int hidden, int n_hidden, int out_dim,
                                uint64_t seed, lhmm_closure_t* out);
lhmm_status lhmm_closure_destroy(lhmm_closure_t c);
/* host arrays: in_mean, in_std (in_dim), out_scale (out_dim); std, scale > 0 */
lhmm_status lhmm_closure_set_normalization(lhmm_closure_t c, const float* in_mean_host,
                                           const float* in_std_host, const float* out_scale_host);
/* One training step of every member: mean-squared error of the scaled
 * outputs against T on the member's own batch, gradient, then AdamW
 * (beta 0.9/0.999, eps 1e-8, decoupled weight decay on weights only) when
 * lr > 0 (lr = 0: gradient only, see lhmm_closure_get_grad).
 *   X_dev     device, rows x in_dim float (the sample table)
 *   T_dev     device, rows x out_dim float (targets, stress units)
 *   rows_dev  device, members x B int row indices into X/T, or NULL to use
 *             rows 0..B-1 for every member
 *   B         batch, a multiple of 32
 *   loss_dev  device, members float (this step's loss per member) or NULL
 * Asynchronous; grows the activation workspace on first use of a batch size. */
lhmm_status lhmm_closure_train_step(lhmm_closure_t c, const float* X_dev, const float* T_dev,
                                    const int* rows_dev, int B, float lr, float weight_decay,
                                    float* loss_dev, void* stream);
/* Ensemble prediction for n inputs: mean_dev n x out_dim (target units) and
 * spread_dev n = sample standard deviation over members of the output vector
 * (Euclidean).  Asynchronous. */
lhmm_status lhmm_closure_infer(lhmm_closure_t c, const float* X_dev, int n, float* mean_dev,
                               float* spread_dev, void* stream);
/* Raw scaled outputs of every member (members x n x out_dim, host).  Sync. */
lhmm_status lhmm_closure_forward(lhmm_closure_t c, const float* X_dev, int n, float* Y_host);
/* Parameters (and last gradient) of one member as host float arrays in the
 * layout W_0, b_0, W_1, b_1, ... with W_l row-major (out x in).  Synchronous. */
lhmm_status lhmm_closure_get_params(lhmm_closure_t c, int member, float* host);
lhmm_status lhmm_closure_set_params(lhmm_closure_t c, int member, const float* host);
lhmm_status lhmm_closure_get_grad(lhmm_closure_t c, int member, float* host);
lhmm_status lhmm_closure_info(lhmm_closure_t c, int64_t* n_params_per_member, int64_t* steps);
/* Tensor-core path of the closure's products: 1 (the default) runs them on
 * the fifth-generation tensor cores (tcgen05.mma with the accumulator in
 * tensor memory, operands staged by TMA); 0 on the warp-level mma.sync path
 * kept for comparison.  Both take BF16 operands and accumulate in FP32, so
 * they differ only by the order of the FP32 sums.  Other values return
 * LHMM_ERR_ARG. */
lhmm_status lhmm_closure_set_gemm(lhmm_closure_t c, int path);
/* Wait for the device; returns LHMM_ERR_TIMEOUT (and clears it) if a
 * tensor-core product gave up a bounded wait since the last call, which
 * leaves its outputs undefined.  Synchronous. */
lhmm_status lhmm_closure_sync(lhmm_closure_t c);

/* ------------------------------------------------------------------------
 * Surrogate-gated macro step (not in the paper).  With a closure attached,
 * every macro step pushes each particle's gradient (Lxx, Lxy, Lyx, Lyy) into a
 * 16-deep ring and builds the closure input [16 past gradients oldest first,
 * pi_xx, pi_xy, pi_yy] (67 floats).  With the gate enabled, a macro step then
 * runs the ensemble; a particle whose ensemble spread exceeds
 * threshold x max(|predicted in-plane stress tensor| (Frobenius), stress_floor)
 * -- or every audit_every-th trusted particle, round robin --
 * runs its DPD box (persistent launch over the device-built list); the others
 * keep their boxes frozen and take pi += predicted increment.  Audited boxes
 * measure the surrogate's live error against DPD.
 * ------------------------------------------------------------------------ */
/* Attach a closure (67 inputs, 3 outputs: increments of pi_xx, pi_xy, pi_yy);
 * the gate starts disabled.  Synchronous; allocates the gate buffers. */
lhmm_status lhmm_coupled_set_closure(lhmm_coupled_t c, lhmm_closure_t closure, float threshold,
                                     float stress_floor, int audit_every);
lhmm_status lhmm_coupled_enable_gate(lhmm_coupled_t c, int enabled);
/* Change the gate's threshold, audit period and target without touching its
 * state (gradient history, counters); threshold and audit_every follow the
 * rules of set_closure.  absolute = 0: the closure predicts the increment of
 * (pi_xx, pi_xy, pi_yy) over the macro step and a trusted particle takes
 * pi += prediction (the set_closure default); absolute = 1: the closure
 * predicts the stress itself from the gradient history alone (the three
 * stress inputs are written as zero), a trusted particle takes pi =
 * prediction, and the relative spread is taken against the predicted stress.
 * Other values return LHMM_ERR_ARG.  warmup_steps: a box that was frozen
 * (trusted) in the previous gated macro step and runs DPD in this one first
 * runs warmup_steps DPD steps under the current gradient whose stress is
 * discarded, then the k' sampled steps; -1 means k' (the default after
 * set_closure), 0 resumes at once; below -1 returns LHMM_ERR_ARG.  The next
 * macro step re-captures its graph.  Synchronous. */
lhmm_status lhmm_coupled_set_gate(lhmm_coupled_t c, float threshold, int audit_every,
                                  int absolute, int warmup_steps);
/* Online calibration of the closure from its audits (not in the paper).  The
 * audited boxes run DPD anyway; after each gated macro step their raw
 * predictions p and DPD values d (per component: the stress in the absolute
 * mode, its increment otherwise) join decayed sums (older steps weighted by
 * decay^age) and a least-squares line d = a p + c is refitted per component
 * (a held to [1/4, 4]; the identity until 20 weighted audits have been
 * seen).  enabled = 1: trusted boxes take a p + c instead of p; 0: they take
 * p (the sums are still kept); -1: change nothing.  decay in (0, 1].
 * map_host (6 floats, or NULL) receives the current (a, c) of xx, xy, yy.
 * The next macro step re-captures its graph.  Synchronous. */
lhmm_status lhmm_coupled_set_online_calibration(lhmm_coupled_t c, int enabled, float decay,
                                                float* map_host);
/* Counters since the closure was attached: gated macro steps, boxes advanced
 * by DPD in them, audited boxes, and over the audited boxes the summed squared
 * error of the predicted increment and the summed squared DPD increment.
 * Synchronous. */
lhmm_status lhmm_coupled_gate_stats(lhmm_coupled_t c, int64_t* gated_steps, int64_t* dpd_boxes,
                                    int64_t* audited_boxes, double* audit_err2, double* audit_ref2);
/* The closure inputs of the last macro step (n_boxes x 67, host).  Sync. */
lhmm_status lhmm_coupled_closure_inputs(lhmm_coupled_t c, float* X_host);

/* ------------------------------------------------------------------------
 * Allocation-free SPH velocity gradient.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory when
 * they need the gradients (code inside another framework's memory pool or an
 * allocator-free real-time section, plug-ins restricted to buffers they are
 * handed).  It computes what lhmm_sph_step(h, ..., n_substeps = 0, L_out) computes
 * for the given particles -- number densities, then L_ab = dv_a/dx_b of every
 * fluid particle -- without a handle and without any allocation: its scratch
 * (cell list, densities, pressures; about 1.5 MiB) is one fixed array in the
 * library's device memory, held by every GPU that loads the library until the
 * process exits.
 *   params     host; n, n_wall, Lx, Ly, h, mass, rho0, c, theta_pb, kernel are
 *              used (the walls are the last n_wall particles).
 *   pos_dev    device, n x 2 float, 8-byte aligned; vel_dev likewise.  Positions
 *              may lie outside [0,Lx) x [0,Ly): each is binned at its periodic
 *              image, and pair distances are minimum-image distances.
 *   L_out_dev  device, (n - n_wall) x 9 float (the lhmm_micro_advance layout).
 * Returns LHMM_ERR_ARG for n > LHMM_NOALLOC_MAX_PARTICLES or more than
 * LHMM_NOALLOC_MAX_CELLS cells (floor(Lx/h) x floor(Ly/h), at least 3 each).
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress).  With lazy module loading (CUDA_MODULE_LOADING=LAZY,
 * the default of recent CUDA runtimes) that lookup may load the library's
 * SPH module, and loading a module is when the driver places the array in
 * device memory.  So make the first call on each device early -- before any
 * stream capture and before any section in which nothing may allocate;
 * later calls allocate nothing.
 * Every call uses the same scratch array, so calls that can overlap on the GPU
 * (different streams, or different host threads) race: serialise them.
 * Asynchronous on `stream`. */
#define LHMM_NOALLOC_MAX_PARTICLES 65536
#define LHMM_NOALLOC_MAX_CELLS 65536
lhmm_status lhmm_sph_velgrad_noalloc(const lhmm_sph_params* params, const float* pos_dev,
                                     const float* vel_dev, float* L_out_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LHMM_H */
