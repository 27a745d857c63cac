// micro.cu -- batched DPD/FENE micro-domains of the LHMM (arXiv 2512.13267,
// Sec. 2.3 and 3.4-3.5, coupling protocol Steps 2-4) on sm_103a.
//
// Design: one thread block owns one box for a whole lhmm_micro_advance call.
// The box's state (cell-relative FP32 positions, velocities, forces, cell ids)
// is loaded once with float4 loads, stays in shared memory for all k' steps,
// and is written back once, so HBM traffic is amortised over k' and the
// kernel is bound by on-chip arithmetic.  Every step the block
//   A  half-kicks and drifts its beads, re-normalising cell-relative offsets
//      and applying Lees-Edwards re-entry (Sec. 2.3 VV; coupling Step 3),
//      and counts each bead into its cell;
//   B  turns the counts into a counting-sort cell list (cells >= rc wide)
//      ordered by (x, id) inside each cell, so every row of cells is sorted
//      by x;
//   C  sums DPD conservative, dissipative and random pair forces (Eqs.
//      conservative, dissipative, random) over the upper half of the 27
//      neighbour cells, each neighbour row cut to the x window that the
//      bead's y, z distance to the row leaves inside rc, accumulating the
//      pair virial of the IK potential stress (Eq. potential_stress) with
//      the core bond fraction;
//   D  per bead: adds its FENE bonds (Eq. fene_force; each bond is computed
//      by both of its beads, its virial by the lower one), half-kicks,
//      imposes v = lambda* L r' on the AFBC BC shell (Eq. micro_bc) and
//      accumulates the IK kinetic stress (Eq. kinetic_stress); then the
//      block reduces the step's stress; the time average (N'_t = k') is
//      kept in FP64.
// Each pair is evaluated once (Newton's third law); pair forces accumulate in
// 2^-18 fixed point with integer shared-memory atomics, which is exact and
// order-independent, so a step is bit-reproducible.  The random term
// theta_ij = theta_ji comes from Philox4x32-10 keyed by the box and counted
// by (min id, max id, step), so it is identical from both sides and across
// runs, and a checkpointed state resumes bit for bit.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "lhmm_common.cuh"

namespace {

struct BoxInfo {
  long long off;      // first bead of the box in the flat arrays
  int n;              // beads
  int n_poly;         // beads in chains (n_chains * chain_len)
  int nc[3];          // cells per axis (>= 3)
  int ncell;
  float w[3];         // cell widths (>= rc)
  float winv[3];
  float len[3];       // periodic lengths nc * w
  float half_core[3]; // AFBC core half widths
  float half_bc[3];   // AFBC BC-shell outer half widths
  float inv_vcore;    // 1 / volume over which IK averages
};

struct BoxState {
  unsigned long long step;  // completed steps; keys the random stream
  float le_offset;          // Lees-Edwards image offset in x, [0, len_x)
  unsigned status;          // LHMM_BOX_* bits
};

struct MicroArgs {
  const BoxInfo* boxes;
  BoxState* state;
  float4* pos;  // (ox, oy, oz, cell id as int bits)
  float4* vel;
  float4* frc;
  const int* list;  // blocks -> box ids
  const float* L;   // n_boxes x 9
  double* stress;
  double* stress_sq;
  int n_steps;
  int init_forces;
  float a, gamma, sig_dt, rc, rc2, rcinv, H, R0, inv_R0sq, dt, hdt_m, mass, lambda_star;
  double out_scale;
  unsigned seed_lo, seed_hi;
  int flow, dpd_on_bonded, chain_len;
  int n_rows;                // rows of the upper half-stencil: 5 in 3D, 2 in 2D
  int excl;                  // DPD pairs of one chain up to excl bonds apart are skipped
  int afbc_peculiar;         // BC beads keep their velocity about their cell's BC mean
  int max_beads, max_cells;
  int n_boxes;
  int id_base;               // random-stream id of box 0 (lhmm_batch_desc.box_id_offset)
  int* work_counter;         // persistent mode: next work item (NULL: one block per item)
  const int* n_items_dev;    // persistent mode: device-side item count
  int max_items;             // persistent mode: capacity of the item list
  int count_lo, count_hi;    // persistent mode: run only if count_lo < item count <= count_hi
  unsigned char* gm;         // boxes held in global memory: per-box scratch (else NULL)
  size_t gm_stride;          // bytes of scratch per box
};

constexpr int kRedFloats = 192;  // 6 x 32 warps, also scan scratch
// Fixed-point pair-force accumulation: resolution 2^-18 (3.8e-6), each
// contribution bounded by kFixMax, so a bead's sum stays far inside int32.
constexpr float kFixScale = 262144.f;
constexpr float kFixInv = 1.f / 262144.f;
constexpr float kFixMax = 512.f;
constexpr int kQueue = 65;       // pair-queue entries per warp (64 + a slot for misses)

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Memory plan of a box of up to N beads and C cells: the box arrays ...
__host__ __device__ inline size_t micro_box_bytes(int N, int C) {
  size_t b = 9 * sizeof(float) * (size_t)N;    // offsets, velocities, forces (SoA)
  b += 2 * sizeof(unsigned short) * (size_t)N;  // cell id per bead, sorted slot -> bead
  b = align16(b);
  b += sizeof(unsigned short) * (size_t)(C + 1); // cell start offsets
  b = align16(b);
  b += sizeof(unsigned short) * (size_t)(C + 1); // cell counters (packed in 32-bit words)
  return align16(b);
}

// ... and the per-block buffers of T threads, always in shared memory.
__host__ __device__ inline size_t micro_block_bytes(int T) {
  size_t b = sizeof(unsigned long long) * (size_t)kQueue * (T / 32);  // pair queues
  b += sizeof(float) * kRedFloats;
  b += sizeof(double) * 12;  // FP64 stress sums
  return b;
}

// Shared memory of one block: box arrays and block buffers (GM: a box held
// in global memory, whose arrays live in a per-box scratch buffer in HBM and
// are served by L1/L2; for boxes beyond one SM's shared memory).
__host__ __device__ inline size_t micro_smem_bytes(int N, int C, int T, bool gm = false) {
  return (gm ? 0 : micro_box_bytes(N, C)) + micro_block_bytes(T);
}

__device__ __forceinline__ int wrapi(int c, int n) {
  c += (c < 0) ? n : 0;
  c -= (c >= n) ? n : 0;
  return c;
}

// Length fraction of segment a->b inside the open box |x_k| < h[k]: the IK
// bond function for a uniform weight on the core (times V_core).
__device__ __forceinline__ float seg_fraction(float ax, float ay, float az, float bx, float by,
                                              float bz, const float* h) {
  float lo = 0.f, hi = 1.f;
  const float a[3] = {ax, ay, az}, d[3] = {bx - ax, by - ay, bz - az};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    // parameter interval of the slab |a + s d| < h (approximate reciprocal:
    // the weight needs a few ulp, not a correctly rounded quotient)
    const bool flat = d[k] == 0.f;
    const float inv = __fdividef(1.f, flat ? 1.f : d[k]);
    const float s1 = (-h[k] - a[k]) * inv, s2 = (h[k] - a[k]) * inv;
    const bool in = fabsf(a[k]) < h[k];
    lo = fmaxf(lo, flat ? (in ? 0.f : 2.f) : fminf(s1, s2));
    hi = fminf(hi, flat ? (in ? 1.f : -1.f) : fmaxf(s1, s2));
  }
  return hi > lo ? hi - lo : 0.f;
}

// A queued pair is one 64-bit word: bead i (bits 0-15), bead j (16-31), the
// x cell offset of j's image relative to i plus 128 (32-39; the offset may
// exceed one cell in a Lees-Edwards shifted row, |offset| < 2 nx + 3 < 128),
// dy + 1 (40-41), dz + 1 (42-43), the IK bond-weight mode of i (44-45) and
// the Lees-Edwards crossing of the row (46-47).
constexpr int kDcxBias = 128;

struct BoxView {
  float *ox, *oy, *oz, *vx, *vy, *vz, *fx, *fy, *fz;
  unsigned short *cellid, *perm, *cstart;
};

// Decode a linear cell index (exact for index < 2^16 in FP32 arithmetic).
__device__ __forceinline__ void cell_coords(int c, int nx, int nxy, float inx, float inxy, int& cx,
                                            int& cy, int& cz) {
  cz = __float2int_rd((static_cast<float>(c) + 0.5f) * inxy);
  const int rem = c - cz * nxy;
  cy = __float2int_rd((static_cast<float>(rem) + 0.5f) * inx);
  cx = rem - cy * nx;
}

// R8's alternative AFBC: per cell, the BC beads keep their velocity about
// the mean velocity of the cell's BC beads, around the imposed field L r'.
// Kept out of line: it runs only in that mode, and inlined it would take
// registers from the pair loop of every mode.
__device__ __noinline__ void afbc_peculiar_pass(float* ox, int NM, const unsigned short* perm,
                                                const unsigned short* cstart, const BoxInfo* B,
                                                const float* sL, int C, int nx, int nxy,
                                                float inx, float inxy) {
  float *oy = ox + NM, *oz = oy + NM, *vx = oz + NM, *vy = vx + NM, *vz = vy + NM;
  const float wx = B->w[0], wy = B->w[1], wz = B->w[2];
  const float hx = 0.5f * B->len[0], hy = 0.5f * B->len[1], hz = 0.5f * B->len[2];
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    int cx, cy, cz;
    cell_coords(c, nx, nxy, inx, inxy, cx, cy, cz);
    const int q0 = cstart[c], q1 = cstart[c + 1];
    float m0 = 0.f, m1 = 0.f, m2 = 0.f;
    int nb = 0;
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = q0; q < q1; ++q) {
        const int i = perm[q];
        const float rpx = static_cast<float>(cx) * wx + ox[i] - hx;
        const float rpy = static_cast<float>(cy) * wy + oy[i] - hy;
        const float rpz = static_cast<float>(cz) * wz + oz[i] - hz;
        const bool core = fabsf(rpx) < B->half_core[0] && fabsf(rpy) < B->half_core[1] &&
                          fabsf(rpz) < B->half_core[2];
        const bool inbc = fabsf(rpx) < B->half_bc[0] && fabsf(rpy) < B->half_bc[1] &&
                          fabsf(rpz) < B->half_bc[2];
        if (core || !inbc) continue;
        if (pass == 0) {
          m0 += vx[i]; m1 += vy[i]; m2 += vz[i];
          ++nb;
        } else {
          vx[i] = sL[0] * rpx + sL[1] * rpy + sL[2] * rpz + (vx[i] - m0);
          vy[i] = sL[3] * rpx + sL[4] * rpy + sL[5] * rpz + (vy[i] - m1);
          vz[i] = sL[6] * rpx + sL[7] * rpy + sL[8] * rpz + (vz[i] - m2);
        }
      }
      if (pass == 0 && nb > 0) {
        const float inv = 1.f / static_cast<float>(nb);
        m0 *= inv; m1 *= inv; m2 *= inv;
      }
    }
  }
}

template <int T, bool PEC, bool GM>
__device__ __forceinline__ void micro_box(const MicroArgs& A, const int bid) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BoxInfo sB;
  __shared__ float sL[9];
  constexpr int NW = T / 32;
  constexpr unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (bid < 0 || bid >= A.n_boxes) return;  // whole block leaves together
  if (tid == 0) sB = A.boxes[bid];
  if (tid < 9) sL[tid] = A.lambda_star * A.L[9 * bid + tid];
  __syncthreads();
  const int N = sB.n, C = sB.ncell;
  const int nx = sB.nc[0], ny = sB.nc[1], nz = sB.nc[2], nxy = nx * ny;
  const float inx = 1.f / static_cast<float>(nx), inxy = 1.f / static_cast<float>(nxy);
  const float wx = sB.w[0], wy = sB.w[1], wz = sB.w[2];

  // carve the box arrays (shared memory, or the box's global scratch) and
  // the block buffers (same plan as micro_smem_bytes)
  const int NM = A.max_beads, CM = A.max_cells;
  unsigned char* const boxmem = GM ? A.gm + static_cast<size_t>(bid) * A.gm_stride : smem;
  BoxView S;
  S.ox = reinterpret_cast<float*>(boxmem);
  S.oy = S.ox + NM;
  S.oz = S.oy + NM;
  S.vx = S.oz + NM;
  S.vy = S.vx + NM;
  S.vz = S.vy + NM;
  S.fx = S.vz + NM;
  S.fy = S.fx + NM;
  S.fz = S.fy + NM;
  S.cellid = reinterpret_cast<unsigned short*>(S.fz + NM);
  S.perm = S.cellid + NM;
  size_t b = align16(9 * sizeof(float) * (size_t)NM + 2 * sizeof(unsigned short) * (size_t)NM);
  S.cstart = reinterpret_cast<unsigned short*>(boxmem + b);
  b = align16(b + sizeof(unsigned short) * (size_t)(CM + 1));
  unsigned* cnt32 = reinterpret_cast<unsigned*>(boxmem + b);  // two 16-bit counters per word
  const unsigned short* cnt16 = reinterpret_cast<const unsigned short*>(cnt32);
  b = align16(b + sizeof(unsigned short) * (size_t)(CM + 1));
  if (GM) b = 0;  // block buffers start the shared memory
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(smem + b) + kQueue * warp;
  b += sizeof(unsigned long long) * (size_t)kQueue * NW;
  float* red = reinterpret_cast<float*>(smem + b);
  float *ox = S.ox, *oy = S.oy, *oz = S.oz, *vx = S.vx, *vy = S.vy, *vz = S.vz;
  float *fx = S.fx, *fy = S.fy, *fz = S.fz;
  unsigned short *cellid = S.cellid, *perm = S.perm, *cstart = S.cstart;
  // pair forces accumulate as 2^-18 fixed point in the force arrays (integer
  // atomics: exact, so the sum does not depend on the order of the adds)
  int* qfx = reinterpret_cast<int*>(fx);
  int* qfy = reinterpret_cast<int*>(fy);
  int* qfz = reinterpret_cast<int*>(fz);

  const long long off = sB.off;
  for (int i = tid; i < N; i += T) {
    const float4 p = A.pos[off + i], v = A.vel[off + i], f = A.frc[off + i];
    ox[i] = p.x; oy[i] = p.y; oz[i] = p.z;
    cellid[i] = static_cast<unsigned short>(__float_as_int(p.w));
    vx[i] = v.x; vy[i] = v.y; vz[i] = v.z;
    fx[i] = f.x; fy[i] = f.y; fz[i] = f.z;
  }

  const bool le = A.flow == LHMM_FLOW_LEES_EDWARDS;
  const bool afbc = A.flow == LHMM_FLOW_AFBC;
  const float gdot = sL[1];                      // LE shear rate (already x lambda*)
  const float vjump = gdot * sB.len[1];          // velocity of the image above
  const float le_inc = vjump * A.dt;             // image offset advance per step
  const unsigned long long step0 = A.state[bid].step;
  const float le0 = A.state[bid].le_offset;
  // key (seed_lo, seed_hi ^ box): distinct (seed, box) pairs with seeds below
  // 2^32 get distinct keys, so consecutive seeds never share a box's noise
  const uint32_t k0 = A.seed_lo, k1 = A.seed_hi ^ static_cast<uint32_t>(A.id_base + bid);
  const float hx = 0.5f * sB.len[0], hy = 0.5f * sB.len[1], hz = 0.5f * sB.len[2];
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned status = 0;
  // FP64 stress sums (component k by thread k) live in shared memory: they
  // would otherwise hold four registers of every thread across the step loop
  double* acc = reinterpret_cast<double*>(red + kRedFloats);
  if (tid < 12) acc[tid] = 0.0;
  // cell counters start at zero; each step's cell pass resets them after use
  for (int c = tid; c < (C + 1) / 2; c += T) cnt32[c] = 0u;
  __syncthreads();
  // a bead's rank in its cell (counting sort) goes to its force word, which
  // is free until the pair pass and reset to zero when the bead is placed
  auto count_in_cell = [&](int i, int c) {
    const unsigned old = atomicAdd(&cnt32[c >> 1], (c & 1) ? 65536u : 1u);
    qfx[i] = (c & 1) ? static_cast<int>(old >> 16) : static_cast<int>(old & 0xffffu);
  };

  const int total_steps = A.init_forces ? 1 : A.n_steps;
  for (int s = 0; s < total_steps; ++s) {
    const bool kick = !A.init_forces;
    const unsigned long long step = kick ? step0 + s + 1 : step0;
    const uint32_t st_lo = static_cast<uint32_t>(step), st_hi = static_cast<uint32_t>(step >> 32);
    float le_off = 0.f;
    if (le) {
      le_off = kick ? le0 + static_cast<float>(s + 1) * le_inc : le0;
      le_off -= floorf(le_off / sB.len[0]) * sB.len[0];
      if (le_off >= sB.len[0]) le_off -= sB.len[0];
    }
    // ---- A: half kick + drift + cell re-normalisation + count into cells
    if (kick) {
      for (int i = tid; i < N; i += T) {
        float v0 = vx[i] + A.hdt_m * fx[i];
        float v1 = vy[i] + A.hdt_m * fy[i];
        float v2 = vz[i] + A.hdt_m * fz[i];
        float o0 = ox[i] + A.dt * v0, o1 = oy[i] + A.dt * v1, o2 = oz[i] + A.dt * v2;
        int cx, cy, cz;
        cell_coords(cellid[i], nx, nxy, inx, inxy, cx, cy, cz);
        if (o1 < 0.f || o1 >= wy) {
          const int k = static_cast<int>(floorf(o1 * sB.winv[1]));
          o1 -= static_cast<float>(k) * wy;
          cy += k;
          if (o1 < 0.f) o1 = 0.f;
          if (o1 >= wy) { o1 -= wy; cy += 1; }
          if (cy >= ny || cy < 0) {
            const int up = cy >= ny;
            cy += up ? -ny : ny;
            if (le) {  // re-enter through the sliding image: shift x, jump v_x
              o0 += up ? -le_off : le_off;
              v0 += up ? -vjump : vjump;
            }
          }
          if (cy < 0 || cy >= ny) {  // moved more than a box in one step
            cy %= ny;
            if (cy < 0) cy += ny;
            status |= LHMM_BOX_NAN;
          }
        }
        if (o0 < 0.f || o0 >= wx) {
          const int k = static_cast<int>(floorf(o0 * sB.winv[0]));
          o0 -= static_cast<float>(k) * wx;
          cx += k;
          if (o0 < 0.f) o0 = 0.f;
          if (o0 >= wx) { o0 -= wx; cx += 1; }
          cx %= nx;
          if (cx < 0) cx += nx;
        }
        if (o2 < 0.f || o2 >= wz) {
          const int k = static_cast<int>(floorf(o2 * sB.winv[2]));
          o2 -= static_cast<float>(k) * wz;
          cz += k;
          if (o2 < 0.f) o2 = 0.f;
          if (o2 >= wz) { o2 -= wz; cz += 1; }
          cz %= nz;
          if (cz < 0) cz += nz;
        }
        ox[i] = o0; oy[i] = o1; oz[i] = o2;
        vx[i] = v0; vy[i] = v1; vz[i] = v2;
        fy[i] = 0.f; fz[i] = 0.f;  // zero bits: fixed-point zero for C
        const int cell = cx + nx * (cy + ny * cz);
        cellid[i] = static_cast<unsigned short>(cell);
        count_in_cell(i, cell);
      }
    } else {
      for (int i = tid; i < N; i += T) {
        fy[i] = 0.f; fz[i] = 0.f;
        count_in_cell(i, cellid[i]);
      }
    }
    __syncthreads();
    // ---- B: counting sort by cell (ranks counted in A)
    {
      const int per = (C + T - 1) / T;
      const int c0 = min(tid * per, C), c1 = min(c0 + per, C);
      int local = 0;
      for (int c = c0; c < c1; ++c) local += cnt16[c];
      int x = local;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
      }
      int* scan = reinterpret_cast<int*>(red);
      if (lane == 31) scan[warp] = x;
      __syncthreads();
      if (warp == 0) {
        int y = lane < NW ? scan[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int z = __shfl_up_sync(FULL, y, o);
          if (lane >= o) y += z;
        }
        if (lane < NW) scan[lane] = y;
      }
      __syncthreads();
      int run = (warp > 0 ? scan[warp - 1] : 0) + x - local;
      for (int c = c0; c < c1; ++c) {
        cstart[c] = static_cast<unsigned short>(run);
        run += cnt16[c];
      }
      if (tid == 0) cstart[C] = static_cast<unsigned short>(scan[NW - 1]);
    }
    __syncthreads();
    for (int i = tid; i < N; i += T) {
      perm[cstart[cellid[i]] + qfx[i]] = static_cast<unsigned short>(i);
      qfx[i] = 0;  // fixed-point zero for C
    }
    __syncthreads();
    for (int c = tid; c < (C + 1) / 2; c += T) cnt32[c] = 0u;  // for the next step
    for (int c = tid; c < C; c += T) {  // ascending (x, id) inside each cell
      const int s0 = cstart[c], s1 = cstart[c + 1];
      for (int p = s0 + 1; p < s1; ++p) {
        const unsigned short key = perm[p];
        const float kx = ox[key];
        int q = p - 1;
        while (q >= s0) {
          const unsigned short o = perm[q];
          const float x = ox[o];
          if (!(x > kx || (x == kx && o > key))) break;
          perm[q + 1] = o;
          --q;
        }
        perm[q + 1] = key;
      }
    }
    __syncthreads();

    // ---- C: forces and pair virial, each pair once (Newton's third law).
    // A lane owns one bead of a work item and scans one row of the upper half
    // of its neighbourhood (its own row after its slot, or one of the rows
    // (dz, dy) = (0,+1), (+1,-1), (+1,0), (+1,+1)), cut to the x window that
    // can hold partners within r_c.  Pairs inside r_c go to the warp's queue
    // and are evaluated 32 at a time with every lane busy; f_i += F_ij and
    // f_j -= F_ij with integer atomics on the box's force words (shared
    // memory, or the box's device scratch in the GM variants).
    float W[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    auto eval_pair = [&](unsigned long long e) {
      const int i = static_cast<int>(e & 0xffffu), j = static_cast<int>((e >> 16) & 0xffffu);
      const int dcx = static_cast<int>((e >> 32) & 0xffu) - kDcxBias;
      const int dy = static_cast<int>((e >> 40) & 3u) - 1, dz = static_cast<int>((e >> 42) & 3u) - 1;
      const int ikm = static_cast<int>((e >> 44) & 3u), cross = static_cast<int>((e >> 46) & 3u);
      const float sx = cross == 1 ? le_off : (cross == 2 ? -le_off : 0.f);
      const float dvs = cross == 1 ? -vjump : (cross == 2 ? vjump : 0.f);
      const float rx = (-static_cast<float>(dcx) * wx - sx) + (ox[i] - ox[j]);
      const float ry = -static_cast<float>(dy) * wy + (oy[i] - oy[j]);
      const float rz = -static_cast<float>(dz) * wz + (oz[i] - oz[j]);
      const float r2 = rx * rx + ry * ry + rz * rz;
      const float rinv = rsqrtf(r2);
      const float r = r2 * rinv;
      const float wR = 1.f - r * A.rcinv;
      const float dvx = vx[i] - vx[j] + dvs, dvy = vy[i] - vy[j], dvz = vz[i] - vz[j];
      const float ev = (rx * dvx + ry * dvy + rz * dvz) * rinv;
      const uint2 rr = lhmm::philox4x32_10_xy(static_cast<uint32_t>(min(i, j)),
                                              static_cast<uint32_t>(max(i, j)), st_lo, st_hi, k0, k1);
      const float th = lhmm::gauss_from_words(rr.x, rr.y);
      const float f = A.a * wR - A.gamma * wR * wR * ev + A.sig_dt * wR * th;
      const float fr = f * rinv;
      float Fx = fr * rx, Fy = fr * ry, Fz = fr * rz;
      if (!(fabsf(Fx) < kFixMax && fabsf(Fy) < kFixMax && fabsf(Fz) < kFixMax)) {
        status |= LHMM_BOX_FORCE_RANGE;  // keep the fixed-point sums in range
        Fx = fminf(fmaxf(Fx, -kFixMax), kFixMax);
        Fy = fminf(fmaxf(Fy, -kFixMax), kFixMax);
        Fz = fminf(fmaxf(Fz, -kFixMax), kFixMax);
        if (Fx != Fx) Fx = 0.f;
        if (Fy != Fy) Fy = 0.f;
        if (Fz != Fz) Fz = 0.f;
      }
      const int ix = __float2int_rn(Fx * kFixScale), iy = __float2int_rn(Fy * kFixScale),
                iz = __float2int_rn(Fz * kFixScale);
      atomicAdd(&qfx[i], ix);
      atomicAdd(&qfy[i], iy);
      atomicAdd(&qfz[i], iz);
      atomicAdd(&qfx[j], -ix);
      atomicAdd(&qfy[j], -iy);
      atomicAdd(&qfz[j], -iz);
      // IK bond weight: 0 outside the core's reach, 1 inside, else the
      // segment fraction (only that case branches)
      float wgt = ikm == 1 ? 1.f : 0.f;
      if (ikm == 2) {
        int cx, cy, cz;
        cell_coords(cellid[i], nx, nxy, inx, inxy, cx, cy, cz);
        const float rpx = static_cast<float>(cx) * wx + ox[i] - hx;
        const float rpy = static_cast<float>(cy) * wy + oy[i] - hy;
        const float rpz = static_cast<float>(cz) * wz + oz[i] - hz;
        wgt = seg_fraction(rpx, rpy, rpz, rpx - rx, rpy - ry, rpz - rz, sB.half_core);
      }
      const float wFx = wgt * Fx, wFy = wgt * Fy, wFz = wgt * Fz;
      W[0] += wFx * rx;
      W[1] += wFy * ry;
      W[2] += wFz * rz;
      W[3] += wFx * ry;
      W[4] += wFx * rz;
      W[5] += wFy * rz;
    };

    // Work items are (chunk of 32 consecutive sorted slots, row) pairs; each
    // warp takes a contiguous share of them, so the block stays balanced when
    // the bead count is not a multiple of the block size.
    int count = 0;  // warp-uniform queue fill
    const int n_rows = A.n_rows;
    const int n_items = n_rows * ((N + 31) >> 5);
    const int per_warp = (n_items + NW - 1) / NW;
    const int it_end = min(n_items, (warp + 1) * per_warp);
    int cur_chunk = -1;
    int k = 0, i = 0, cx = 0, cy = 0, cz = 0, ikm = 1;
    float xi = 0.f, yi = 0.f, zi = 0.f;
    for (int it = warp * per_warp; it < it_end; ++it) {
      const int chunk = it / n_rows, row = it - n_rows * chunk;
      if (chunk != cur_chunk) {  // warp-uniform: load bead k = 32 chunk + lane
        cur_chunk = chunk;
        k = (chunk << 5) + lane;
        const bool own = k < N;
        i = own ? perm[k] : 0;
        cx = cy = cz = 0;
        ikm = 1;
        xi = yi = zi = 0.f;
        if (own) {
          cell_coords(cellid[i], nx, nxy, inx, inxy, cx, cy, cz);
          xi = ox[i]; yi = oy[i]; zi = oz[i];
          if (afbc) {  // a pair segment reaches at most rc from bead i (max norm)
            const float rpx = static_cast<float>(cx) * wx + xi - hx;
            const float rpy = static_cast<float>(cy) * wy + yi - hy;
            const float rpz = static_cast<float>(cz) * wz + zi - hz;
            const float m = fmaxf(fabsf(rpx) - sB.half_core[0],
                                  fmaxf(fabsf(rpy) - sB.half_core[1], fabsf(rpz) - sB.half_core[2]));
            ikm = (m >= A.rc) ? 0 : ((m < -A.rc) ? 1 : 2);
          }
        }
      }
      {
        // upper-half rows of cells: (dz, dy) = (0,0) [slots after k up to
        // x_i + rc], (0,+1), (+1,-1), (+1,0), (+1,+1) [an x window each]
        const int dz = row < 2 ? 0 : 1;
        const int dy = row == 0 ? 0 : (row == 1 ? 1 : row - 3);
        // The window is one run of slots in unwrapped row order: candidate t
        // (0 <= t < len) is slot s + t, or s + t - (row length) from t = tj on
        // when the window wraps around the row end.  The run covers at most
        // three x cells (unwrapped: c0, c0 + 1, c0 + 2, starting at t = 0,
        // t0, t1); xb = x_i - dc*wx - shift with dc the x cell offset of c0
        // (j's image relative to i), so rx = xb - wx*[(t >= t0) + (t >= t1)]
        // - ox[j], and hw is the upper word of a queue entry in cell c0.
        int s = 0, sw = 0, tj = 0x7fffffff, len = 0, t0 = 0, t1 = 0;
        float xb0 = 0.f, xb1 = 0.f, xb2 = 0.f;
        unsigned hw0 = 0u;
        const int z = wrapi(cz + dz, nz);
        int y = cy + dy;
        const bool below = y < 0, above = y >= ny;
        y += below ? ny : (above ? -ny : 0);
        const int cross = !le ? 0 : (below ? 2 : (above ? 1 : 0));
        const float sxr = !le ? 0.f : (below ? -le_off : (above ? le_off : 0.f));
        // Beads of the row's cell column within rc of i lie within |x_j - c|
        // < w of the (image-shifted) centre c = x_i - sxr, where w^2 = rc^2 -
        // ey^2 - ez^2 and ey, ez are i's distances to the column in y and z;
        // the row is sorted by x, so the candidates are one slot window (two
        // where it wraps around the row).
        const float ey = dy > 0 ? wy - yi : (dy < 0 ? yi : 0.f);
        const float ez = dz > 0 ? wz - zi : 0.f;
        const float w2 = A.rc2 - ey * ey - ez * ez;
        // computed by every lane (no divergent branch); lanes without a
        // window (past the last bead, or w^2 <= 0) get zero lengths at the end
        const bool has_window = k < N && w2 > 0.f;
        {
          const float lenx = sB.len[0], winvx = sB.winv[0];
          const float xa = static_cast<float>(cx) * wx + xi;
          const unsigned hiw = (static_cast<unsigned>(dy + 1) << 8) |
                               (static_cast<unsigned>(dz + 1) << 10) |
                               (static_cast<unsigned>(ikm) << 12) |
                               (static_cast<unsigned>(cross) << 14);
          const int rowbase = nx * (y + ny * z);
          // first slot of the row with x >= X (X in [0, lenx]) and the cell
          // that holds X: inside the cell (sorted by x) the length of the
          // prefix with x < X is built from steps of 8, 4, 2, 1 (exact up to
          // 15 beads), then extended one by one (only in cells of more)
          auto lower = [&](float X, int& cell) -> int {
            const int c = min(__float2int_rd(X * winvx), nx - 1);
            const float xr = X - static_cast<float>(c) * wx;
            int lo = cstart[rowbase + c];
            int n = cstart[rowbase + c + 1] - lo;
#pragma unroll
            for (int st = 8; st > 0; st >>= 1) {
              const bool ok = st <= n;  // probe inside the cell, else a valid dummy slot
              const bool take = ok && ox[perm[ok ? lo + st - 1 : 0]] < xr;
              lo += take ? st : 0;
              n -= take ? st : 0;
            }
            while (n > 0 && ox[perm[lo]] < xr) {
              ++lo;
              --n;
            }
            cell = c;
            return lo;
          };
          // window [X0, X1) in unwrapped row coordinates (image m0); the own
          // row starts right after slot k
          float X0 = xa, X1 = xa + A.rc + 1e-5f;
          int m0 = 0;
          if (row != 0) {
            const float w2s = has_window ? w2 : 1e-12f;
            // margin covers rsqrtf's error; capped at the cell width (every
            // true pair has |dx| < rc <= wx), so a window of 2w never reaches
            // a fourth cell, which the two cell-start slots e0, e1 below
            // could not place
            const float w = fminf(w2s * rsqrtf(w2s) + 1e-5f, wx);
            float cc = xa - sxr;  // in (-lenx, 2 lenx)
            const bool neg = cc < 0.f, big = cc >= lenx;
            cc = neg ? cc + lenx : (big ? cc - lenx : cc);
            m0 = neg ? -1 : (big ? 1 : 0);
            X0 = cc - w;
            X1 = cc + w;
          }
          const bool wl = X0 < 0.f, wh = X1 > lenx, wrap = wl || wh;
          int c0 = cx, c1;
          const int q0 = (row == 0) ? k + 1 : lower(wl ? X0 + lenx : X0, c0);
          const int q1 = lower(wh ? X1 - lenx : X1, c1);
          const int rowstart = cstart[rowbase], rowend = cstart[rowbase + nx];
          const int dc = c0 + (wl ? m0 - 1 : m0) * nx - cx;
          s = q0;
          sw = q0 - (rowend - rowstart);
          tj = wrap ? rowend - q0 : 0x7fffffff;
          len = wrap ? (rowend - q0) + (q1 - rowstart) : max(q1 - q0, 0);
          len = has_window ? len : 0;
          // slot offsets of the next two cells (past the row end: the row's
          // first cells, one image on)
          t0 = cstart[rowbase + c0 + 1] - q0;
          t1 = (c0 + 2 <= nx ? cstart[rowbase + c0 + 2] : rowend + cstart[rowbase + 1] - rowstart) - q0;
          xb0 = (-static_cast<float>(dc) * wx - sxr) + xi;
          xb1 = xb0 - wx;
          xb2 = xb1 - wx;
          hw0 = hiw + static_cast<unsigned>(dc + kDcxBias);
        }
        const int lmax = __reduce_max_sync(FULL, len);
        const float yb = -static_cast<float>(dy) * wy + yi, zb = -static_cast<float>(dz) * wz + zi;
        const unsigned lo_i = static_cast<unsigned>(i);
        // fill the warp's queue from the slot windows; whenever it holds 32
        // pairs, leave the (register-light) fill loop to evaluate them
        int t = 0;
        while (true) {
          for (; t < lmax && count < 32; ++t) {
            bool hit;
            unsigned lo_w, hi_w;
            {  // no divergent branch: lanes past their window test slot 0
              const bool act = t < len;
              const bool p0 = t >= t0, p1 = t >= t1;
              int q = t + (t >= tj ? sw : s);
              q = act ? q : 0;
              const float bx = p1 ? xb2 : (p0 ? xb1 : xb0);
              const int j = perm[q];
              const float rx = bx - ox[j];
              const float ry = yb - oy[j];
              const float rz = zb - oz[j];
              const float r2 = rx * rx + ry * ry + rz * rz;
              hit = act && (r2 < A.rc2) && (r2 > 0.f);
              if (A.excl > 0) {  // uniform: pairs of one chain <= excl bonds apart skip DPD
                const int lo = min(i, j), d = max(i, j) - lo;
                hit = hit && !(d <= A.excl && lo + d < sB.n_poly && (lo % A.chain_len) + d < A.chain_len);
              }
              lo_w = lo_i | (static_cast<unsigned>(j) << 16);
              hi_w = hw0 + static_cast<unsigned>(p0) + static_cast<unsigned>(p1);
            }
            const unsigned bal = __ballot_sync(FULL, hit);
            // every lane stores (no divergent branch): misses go to the spare
            // last slot, which no entry ever occupies (count + 32 <= 63)
            queue[hit ? count + __popc(bal & lt_mask) : kQueue - 1] =
                (static_cast<unsigned long long>(hi_w) << 32) | lo_w;
            count += __popc(bal);
          }
          if (count < 32) break;
          __syncwarp();
          eval_pair(queue[lane]);
          __syncwarp();
          queue[lane] = queue[32 + lane];  // entries past count - 32 are dead
          __syncwarp();
          count -= 32;
        }
      }
    }
    __syncwarp();
    if (lane < count) eval_pair(queue[lane]);
    __syncthreads();
    // FENE bonds (k, k+1) inside a chain, attractive (Eq. fene_force): the
    // bond vector and force of bond k, computed the same way by both of its
    // beads, so each bead sums its own forces without atomics or a barrier
    auto fene = [&](int k, float& Fx, float& Fy, float& Fz, float& rx, float& ry, float& rz,
                    int& cxk, int& cyk, int& czk) {
      const int j = k + 1;
      int cxj, cyj, czj;
      cell_coords(cellid[k], nx, nxy, inx, inxy, cxk, cyk, czk);
      cell_coords(cellid[j], nx, nxy, inx, inxy, cxj, cyj, czj);
      rx = static_cast<float>(cxk - cxj) * wx + (ox[k] - ox[j]);
      ry = static_cast<float>(cyk - cyj) * wy + (oy[k] - oy[j]);
      rz = static_cast<float>(czk - czj) * wz + (oz[k] - oz[j]);
      if (ry > hy) {
        ry -= sB.len[1];
        if (le) rx -= le_off;
      } else if (ry < -hy) {
        ry += sB.len[1];
        if (le) rx += le_off;
      }
      rx -= sB.len[0] * rintf(rx / sB.len[0]);
      if (rz > hz) rz -= sB.len[2];
      else if (rz < -hz) rz += sB.len[2];
      float x = (rx * rx + ry * ry + rz * rz) * A.inv_R0sq;
      if (!(x < 1.f)) {
        status |= LHMM_BOX_BOND_OVERSTRETCH;
        x = 0.99f;
      }
      const float cf = -A.H / (1.f - x);
      Fx = cf * rx;
      Fy = cf * ry;
      Fz = cf * rz;
    };
    // ---- D: per bead: pair forces (fixed point -> FP32) plus its bonds,
    // second half kick, AFBC imposition, IK kinetic part
    for (int i = tid; i < N; i += T) {
      float f0 = static_cast<float>(qfx[i]) * kFixInv;
      float f1 = static_cast<float>(qfy[i]) * kFixInv;
      float f2 = static_cast<float>(qfz[i]) * kFixInv;
      if (i < sB.n_poly) {
        const int c = i % A.chain_len;
        float up0 = 0.f, up1 = 0.f, up2 = 0.f, dn0 = 0.f, dn1 = 0.f, dn2 = 0.f;
        if (c + 1 < A.chain_len) {  // bond (i, i+1): +F on i, and its virial
          float Fx, Fy, Fz, rx, ry, rz;
          int cxk, cyk, czk;
          fene(i, Fx, Fy, Fz, rx, ry, rz, cxk, cyk, czk);
          up0 = Fx; up1 = Fy; up2 = Fz;
          float wgt = 1.f;
          if (afbc) {  // a bond is shorter than R0
            const float rpx = static_cast<float>(cxk) * wx + ox[i] - hx;
            const float rpy = static_cast<float>(cyk) * wy + oy[i] - hy;
            const float rpz = static_cast<float>(czk) * wz + oz[i] - hz;
            const float m = fmaxf(fabsf(rpx) - sB.half_core[0],
                                  fmaxf(fabsf(rpy) - sB.half_core[1], fabsf(rpz) - sB.half_core[2]));
            if (m >= A.R0) wgt = 0.f;
            else if (m >= -A.R0)
              wgt = seg_fraction(rpx, rpy, rpz, rpx - rx, rpy - ry, rpz - rz, sB.half_core);
          }
          W[0] += wgt * Fx * rx;
          W[1] += wgt * Fy * ry;
          W[2] += wgt * Fz * rz;
          W[3] += wgt * Fx * ry;
          W[4] += wgt * Fx * rz;
          W[5] += wgt * Fy * rz;
        }
        if (c > 0) {  // bond (i-1, i): -F on i
          float Fx, Fy, Fz, rx, ry, rz;
          int cxk, cyk, czk;
          fene(i - 1, Fx, Fy, Fz, rx, ry, rz, cxk, cyk, czk);
          dn0 = Fx; dn1 = Fy; dn2 = Fz;
        }
        // bonds starting at an even bead first, then those at an odd bead
        if ((i & 1) == 0) {
          if (c + 1 < A.chain_len) { f0 += up0; f1 += up1; f2 += up2; }
          if (c > 0) { f0 -= dn0; f1 -= dn1; f2 -= dn2; }
        } else {
          if (c > 0) { f0 -= dn0; f1 -= dn1; f2 -= dn2; }
          if (c + 1 < A.chain_len) { f0 += up0; f1 += up1; f2 += up2; }
        }
      }
      fx[i] = f0; fy[i] = f1; fz[i] = f2;
      if (A.init_forces) continue;
      float v0 = vx[i] + A.hdt_m * f0;
      float v1 = vy[i] + A.hdt_m * f1;
      float v2 = vz[i] + A.hdt_m * f2;
      int cx, cy, cz;
      cell_coords(cellid[i], nx, nxy, inx, inxy, cx, cy, cz);
      const float rpx = static_cast<float>(cx) * wx + ox[i] - hx;
      const float rpy = static_cast<float>(cy) * wy + oy[i] - hy;
      const float rpz = static_cast<float>(cz) * wz + oz[i] - hz;
      bool sample = true;
      float u0 = 0.f, u1 = 0.f, u2 = 0.f;
      if (afbc) {
        const bool core = fabsf(rpx) < sB.half_core[0] && fabsf(rpy) < sB.half_core[1] &&
                          fabsf(rpz) < sB.half_core[2];
        const bool inbc = fabsf(rpx) < sB.half_bc[0] && fabsf(rpy) < sB.half_bc[1] &&
                          fabsf(rpz) < sB.half_bc[2];
        u0 = sL[0] * rpx + sL[1] * rpy + sL[2] * rpz;
        u1 = sL[3] * rpx + sL[4] * rpy + sL[5] * rpz;
        u2 = sL[6] * rpx + sL[7] * rpy + sL[8] * rpz;
        if (!core && inbc && !PEC) {
          v0 = u0; v1 = u1; v2 = u2;
        }
        sample = core;
      } else if (le) {
        u0 = gdot * rpy;
      }
      vx[i] = v0; vy[i] = v1; vz[i] = v2;
      if (sample) {
        const float d0 = v0 - u0, d1 = v1 - u1, d2 = v2 - u2;
        W[0] += A.mass * d0 * d0;
        W[1] += A.mass * d1 * d1;
        W[2] += A.mass * d2 * d2;
        W[3] += A.mass * d0 * d1;
        W[4] += A.mass * d0 * d2;
        W[5] += A.mass * d1 * d2;
      }
    }
    if (A.init_forces) {
      __syncthreads();
      break;
    }
    if (PEC && afbc) {
      __syncthreads();
      afbc_peculiar_pass(ox, NM, perm, cstart, &sB, sL, C, nx, nxy, inx, inxy);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float v = lhmm::warp_sum(W[k]);
      if (lane == 0) red[6 * warp + k] = v;
    }
    __syncthreads();
    if (tid < 6) {
      float sum = 0.f;
      for (int w = 0; w < NW; ++w) sum += red[6 * w + tid];
      const double pi = -static_cast<double>(sum) * static_cast<double>(sB.inv_vcore);
      acc[tid] += pi;
      acc[6 + tid] += pi * pi;
    }
    // no barrier here: `red` is next written by the cell scan, after the
    // barrier that ends the next step's drift, which threads 0..5 reach only
    // after this sum
  }

  // write back
  for (int i = tid; i < N; i += T) {
    const float4 v = make_float4(vx[i], vy[i], vz[i], 0.f);
    const float4 f = make_float4(fx[i], fy[i], fz[i], 0.f);
    if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(f.x) && isfinite(f.y) &&
          isfinite(f.z)))
      status |= LHMM_BOX_NAN;
    A.pos[off + i] = make_float4(ox[i], oy[i], oz[i], __int_as_float(static_cast<int>(cellid[i])));
    A.vel[off + i] = v;
    A.frc[off + i] = f;
  }
  if (status) atomicOr(&A.state[bid].status, status);
  if (!A.init_forces && A.n_steps > 0) {
    if (tid < 6) {
      const double inv = 1.0 / static_cast<double>(A.n_steps);
      A.stress[6 * bid + tid] = A.out_scale * acc[tid] * inv;
      if (A.stress_sq) A.stress_sq[6 * bid + tid] = A.out_scale * A.out_scale * acc[6 + tid] * inv;
    }
    if (tid == 0) {
      A.state[bid].step = step0 + static_cast<unsigned long long>(A.n_steps);
      if (le) {
        float l = le0 + static_cast<float>(A.n_steps) * le_inc;
        l -= floorf(l / sB.len[0]) * sB.len[0];
        if (l >= sB.len[0]) l -= sB.len[0];
        A.state[bid].le_offset = l;
      }
    }
  }
}


// One block per listed box.  PEC: the AFBC shell keeps the beads' peculiar
// velocity (a separate instantiation, so the other modes' register
// allocation does not carry that pass).  GM: the box arrays live in a
// per-box global scratch buffer instead of shared memory.
template <int T, int MINB, bool PEC, bool GM>
__global__ void __launch_bounds__(T, MINB) micro_kernel(const MicroArgs A) {
  micro_box<T, PEC, GM>(A, A.list[blockIdx.x]);
}

// Persistent form: a fixed grid whose blocks pull item indices from a device
// counter up to a device-side count, so the set of boxes can be chosen on the
// device (e.g. by a gate inside a CUDA graph).
template <int T, int MINB, bool PEC, bool GM>
__global__ void __launch_bounds__(T, MINB) micro_kernel_persistent(const MicroArgs A) {
  __shared__ int s_item;
  {
    // a launch shaped for another range of item counts leaves the items to
    // it (the same test in every thread, before any barrier)
    const int count = min(*A.n_items_dev, A.max_items);
    if (count <= A.count_lo || count > A.count_hi) return;
  }
  for (;;) {
    if (threadIdx.x == 0) {
      const int item = atomicAdd(A.work_counter, 1);
      s_item = item < min(*A.n_items_dev, A.max_items) ? item : -1;
    }
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item < 0) return;
    micro_box<T, PEC, GM>(A, A.list[item]);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Conserved-quantity diagnostics (Eq. motion without its dissipative and
// random terms conserves momentum and the energy below).  One block per box
// reads the resident state and sums in FP64: total momentum sum m v, kinetic
// energy sum m v^2 / 2, the conservative DPD potential U = a rc/2 (1 -
// r/rc)^2 of every non-excluded pair within rc (the potential of Eq.
// conservative), and the FENE potential -H R0^2/2 ln(1 - r^2/R0^2) of every
// bond (Eq. fene_force).  Pairs are found by brute force over the box in a
// balanced half ring (bead i meets i+1 .. i+N/2 mod N), displacements are
// formed from the cell-relative positions with the minimum image (Lees-
// Edwards shifted across y), so the result does not depend on the cell list.
constexpr int kDiagThreads = 256;

__device__ __forceinline__ void diag_disp(const BoxInfo& B, float le_off, bool le, float4 a,
                                          float4 b, float& rx, float& ry, float& rz) {
  const int ca = __float_as_int(a.w), cb = __float_as_int(b.w);
  const int nx = B.nc[0], nxy = B.nc[0] * B.nc[1];
  const int az = ca / nxy, ay = (ca - az * nxy) / nx, ax = ca - az * nxy - ay * nx;
  const int bz = cb / nxy, by = (cb - bz * nxy) / nx, bx = cb - bz * nxy - by * nx;
  rx = static_cast<float>(ax - bx) * B.w[0] + (a.x - b.x);
  ry = static_cast<float>(ay - by) * B.w[1] + (a.y - b.y);
  rz = static_cast<float>(az - bz) * B.w[2] + (a.z - b.z);
  if (ry > 0.5f * B.len[1]) {
    ry -= B.len[1];
    if (le) rx -= le_off;
  } else if (ry < -0.5f * B.len[1]) {
    ry += B.len[1];
    if (le) rx += le_off;
  }
  rx -= B.len[0] * rintf(rx / B.len[0]);
  rz -= B.len[2] * rintf(rz / B.len[2]);
}

__global__ void __launch_bounds__(kDiagThreads) micro_diagnostics_kernel(const MicroArgs A,
                                                                         double* out) {
  __shared__ double red[kDiagThreads / 32][7];
  const int bid = blockIdx.x;
  const BoxInfo B = A.boxes[bid];
  const bool le = A.flow == LHMM_FLOW_LEES_EDWARDS;
  const float le_off = A.state[bid].le_offset;
  const float4* pos = A.pos + B.off;
  const float4* vel = A.vel + B.off;
  const int N = B.n;
  double s[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  bool over = false;
  const float rc2 = A.rc * A.rc;
  for (int i = threadIdx.x; i < N; i += kDiagThreads) {
    const float4 v = vel[i];
    const double m = static_cast<double>(A.mass);
    s[0] += m * v.x;
    s[1] += m * v.y;
    s[2] += m * v.z;
    s[3] += 0.5 * m * (static_cast<double>(v.x) * v.x + static_cast<double>(v.y) * v.y +
                       static_cast<double>(v.z) * v.z);
    const float4 pi = pos[i];
    // half ring: i meets i+1 .. i+N/2 (mod N); with N even, the partner at
    // distance N/2 is taken by the lower bead only
    const int half = N / 2;
    const int last = (N % 2 == 0 && i >= half) ? half - 1 : half;
    for (int k = 1; k <= last; ++k) {
      int j = i + k;
      j -= (j >= N) ? N : 0;
      float rx, ry, rz;
      diag_disp(B, le_off, le, pi, __ldg(&pos[j]), rx, ry, rz);
      const float r2 = rx * rx + ry * ry + rz * rz;
      if (r2 < rc2) {
        const int lo = min(i, j), d = max(i, j) - lo;
        const bool excl = A.excl > 0 && d <= A.excl && lo + d < B.n_poly &&
                          (lo % A.chain_len) + d < A.chain_len;
        if (!excl) {
          const double w = 1.0 - sqrt(static_cast<double>(r2)) / static_cast<double>(A.rc);
          s[4] += 0.5 * static_cast<double>(A.a) * static_cast<double>(A.rc) * w * w;
        }
      }
    }
    if (i + 1 < B.n_poly && (i + 1) % A.chain_len != 0) {  // bond (i, i+1)
      float rx, ry, rz;
      diag_disp(B, le_off, le, pi, pos[i + 1], rx, ry, rz);
      double x = (static_cast<double>(rx) * rx + static_cast<double>(ry) * ry +
                  static_cast<double>(rz) * rz) / (static_cast<double>(A.R0) * A.R0);
      if (!(x < 1.0)) {
        x = 0.99;
        over = true;
      }
      s[5] += -0.5 * static_cast<double>(A.H) * static_cast<double>(A.R0) * A.R0 * log(1.0 - x);
    }
  }
  s[6] = over ? 1.0 : 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    double v = s[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double v = 0.0;
    for (int w = 0; w < kDiagThreads / 32; ++w) v += red[w][threadIdx.x];
    red[0][threadIdx.x] = v;  // each thread rewrites only its own column
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double* o = out + 8 * bid;
    o[0] = red[0][0];
    o[1] = red[0][1];
    o[2] = red[0][2];
    o[3] = red[0][3];
    o[4] = red[0][4];
    o[5] = red[0][5];
    o[6] = red[0][3] + red[0][4] + red[0][5];
    o[7] = red[0][6] > 0.0 ? 1.0 : 0.0;
  }
}

// Launch variants: threads per block and the resident blocks per SM that
// the register allocation must allow (64 registers/thread for 2048/SM).
struct Variant {
  int threads, min_blocks;
  bool gm;  // box arrays in global scratch (boxes beyond one SM's shared memory)
};
constexpr Variant kVariants[] = {{256, 4, false}, {512, 2, false}, {1024, 1, false},
                                 {256, 2, false}, {512, 1, false}, {512, 1, true},
                                 {256, 2, true}};
constexpr int kFirstGmVariant = 5;
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
static_assert(kNumVariants == LHMM_MICRO_N_VARIANTS, "variant table and header disagree");

template <int T, int MINB, bool PEC, bool GM>
cudaError_t launch_micro_mode(const MicroArgs& a, int grid, size_t smem, cudaStream_t s) {
  static size_t attr_bytes = 0, attr_bytes_p = 0;
  const bool persistent = a.work_counter != nullptr;
  size_t& done = persistent ? attr_bytes_p : attr_bytes;
  if (smem > done) {
    cudaError_t e = persistent
                        ? cudaFuncSetAttribute(micro_kernel_persistent<T, MINB, PEC, GM>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem))
                        : cudaFuncSetAttribute(micro_kernel<T, MINB, PEC, GM>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    done = smem;
  }
  if (persistent) micro_kernel_persistent<T, MINB, PEC, GM><<<grid, T, smem, s>>>(a);
  else micro_kernel<T, MINB, PEC, GM><<<grid, T, smem, s>>>(a);
  return cudaGetLastError();
}

template <int T, int MINB, bool GM = false>
cudaError_t launch_micro(const MicroArgs& a, int grid, size_t smem, cudaStream_t s) {
  return a.afbc_peculiar ? launch_micro_mode<T, MINB, true, GM>(a, grid, smem, s)
                         : launch_micro_mode<T, MINB, false, GM>(a, grid, smem, s);
}

cudaError_t launch_variant(int v, const MicroArgs& a, int grid, size_t smem, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  if (kVariants[v].gm && a.gm == nullptr) return cudaErrorInvalidValue;
  switch (v) {
    case 0: return launch_micro<256, 4>(a, grid, smem, s);
    case 1: return launch_micro<512, 2>(a, grid, smem, s);
    case 2: return launch_micro<1024, 1>(a, grid, smem, s);
    case 3: return launch_micro<256, 2>(a, grid, smem, s);
    case 4: return launch_micro<512, 1>(a, grid, smem, s);
    case 5: return launch_micro<512, 1, true>(a, grid, smem, s);
    default: return launch_micro<256, 2, true>(a, grid, smem, s);
  }
}

// A size class: boxes of similar bead count launched together with a shared
// memory plan sized to the class, on a stream of its own.
struct SizeClass {
  std::vector<int> boxes;  // host copy, longest first
  int* boxes_d = nullptr;
  int max_beads = 1, max_cells = 1;
  int variant = 1;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

}  // namespace

struct lhmm_micro_s {
  lhmm_dpd_params p;
  int n_boxes = 0, chain_len = 0, max_beads = 0, max_cells = 0;
  int id_base = 0;  // random-stream id of box 0
  long long total = 0;
  std::vector<BoxInfo> info;
  BoxInfo* info_d = nullptr;
  BoxState* state_d = nullptr;
  float4 *pos_d = nullptr, *vel_d = nullptr, *frc_d = nullptr;
  int* order_d = nullptr;
  float* L_stage = nullptr;
  double *st_stage = nullptr, *sq_stage = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<SizeClass> classes;
  cudaEvent_t fork = nullptr;
  int* work_counter = nullptr;  // persistent-mode item counter
  bool all_persistent = false;  // full advances as one persistent launch (autotuner's choice)
  int all_variant = 0;          // its kernel variant
  int* n_all_d = nullptr;       // device copy of n_boxes, its item count
  int subset_variant = 1;   // launches over a box list, at most one box per resident slot
  int list_tp_variant = 1;  // launches over a box list with more boxes than that
  unsigned char* gm = nullptr;  // per-box scratch of the global-memory variants
  size_t gm_stride = 0;
};

namespace {

size_t max_optin_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return static_cast<size_t>(v);
}

size_t class_smem(int max_beads, int max_cells, int variant) {
  return micro_smem_bytes(max_beads, max_cells, kVariants[variant].threads, kVariants[variant].gm);
}

// whether some shared-memory variant holds a class of this size
bool fits_shared(int max_beads, int max_cells, size_t optin) {
  for (int v = 0; v < kFirstGmVariant; ++v)
    if (class_smem(max_beads, max_cells, v) <= optin) return true;
  return false;
}

// per-box global scratch for the GM variants, sized for the largest box
cudaError_t ensure_gm(lhmm_micro_s* h) {
  if (h->gm) return cudaSuccess;
  const size_t stride = micro_box_bytes(h->max_beads, h->max_cells);
  const size_t n = static_cast<size_t>(std::max(h->n_boxes, 1));
  cudaError_t e = cudaMalloc(&h->gm, stride * n);
  if (e != cudaSuccess) {
    h->gm = nullptr;
    return e;
  }
  h->gm_stride = stride;
  return cudaSuccess;
}

// heuristic start: more threads for larger boxes; the autotuner refines it
int default_variant(int n) { return n <= 1100 ? 0 : (n <= 2600 ? 1 : 2); }

// Variant of the launches over a box list (subset and device-list
// advances, which a gated coupled step uses for the few boxes it sends to
// DPD): one box per SM and as many threads as fit, so that a box finishes
// in the fewest clocks; a box that no shared-memory plan holds runs in the
// device-memory variant.
int list_variant(int max_beads, int max_cells, size_t optin) {
  for (int v : {2, 4, 1, 0, 3})
    if (micro_smem_bytes(max_beads, max_cells, kVariants[v].threads, kVariants[v].gm) <= optin)
      return v;
  return kFirstGmVariant;
}

// ... and with more boxes than SMs: two blocks of 512 threads per SM, which
// measured fastest from one to eight boxes per SM (1000- and 1500-bead
// boxes), else the latency shape
int list_tp_variant(int max_beads, int max_cells, size_t optin, int latency_variant) {
  return micro_smem_bytes(max_beads, max_cells, kVariants[1].threads, kVariants[1].gm) <= optin
             ? 1
             : latency_variant;
}

void abs_to_rel(const BoxInfo& B, const double* x, float4* out, int n) {
  for (int i = 0; i < n; ++i) {
    int c[3];
    float o[3];
    for (int a = 0; a < 3; ++a) {
      const double len = B.len[a], w = B.w[a];
      double xa = x[3 * i + a];
      xa -= std::floor(xa / len) * len;
      if (xa >= len) xa -= len;
      if (xa < 0.0) xa = 0.0;
      int ca = static_cast<int>(std::floor(xa / w));
      ca = std::min(std::max(ca, 0), B.nc[a] - 1);
      double oa = xa - static_cast<double>(ca) * w;  // exact for x = c w + o
      if (oa < 0.0) oa = 0.0;
      if (oa > w) oa = w;
      c[a] = ca;
      o[a] = static_cast<float>(oa);
    }
    const int cell = c[0] + B.nc[0] * (c[1] + B.nc[1] * c[2]);
    float cw;
    std::memcpy(&cw, &cell, sizeof(float));
    out[i] = make_float4(o[0], o[1], o[2], cw);
  }
}

void rel_to_abs(const BoxInfo& B, const float4* in, double* x, int n) {
  for (int i = 0; i < n; ++i) {
    int cell;
    std::memcpy(&cell, &in[i].w, sizeof(int));
    const int c[3] = {cell % B.nc[0], (cell / B.nc[0]) % B.nc[1], cell / (B.nc[0] * B.nc[1])};
    const float o[3] = {in[i].x, in[i].y, in[i].z};
    for (int a = 0; a < 3; ++a)
      x[3 * i + a] = static_cast<double>(c[a]) * static_cast<double>(B.w[a]) + static_cast<double>(o[a]);
  }
}

void free_micro(lhmm_micro_t h) {
  if (!h) return;
  cudaFree(h->info_d);
  cudaFree(h->state_d);
  cudaFree(h->pos_d);
  cudaFree(h->vel_d);
  cudaFree(h->frc_d);
  cudaFree(h->order_d);
  cudaFree(h->L_stage);
  cudaFree(h->st_stage);
  cudaFree(h->sq_stage);
  for (auto& c : h->classes) {
    cudaFree(c.boxes_d);
    if (c.stream) cudaStreamDestroy(c.stream);
    if (c.done) cudaEventDestroy(c.done);
  }
  if (h->fork) cudaEventDestroy(h->fork);
  cudaFree(h->work_counter);
  cudaFree(h->n_all_d);
  cudaFree(h->gm);
  delete h;
}

MicroArgs make_args(const lhmm_micro_s* h) {
  MicroArgs a{};
  const lhmm_dpd_params& p = h->p;
  a.boxes = h->info_d;
  a.state = h->state_d;
  a.pos = h->pos_d;
  a.vel = h->vel_d;
  a.frc = h->frc_d;
  a.a = p.a_ij;
  a.gamma = p.gamma;
  a.sig_dt = static_cast<float>(static_cast<double>(p.sigma) / std::sqrt(static_cast<double>(p.dt)));
  a.rc = p.rc;
  a.rc2 = p.rc * p.rc;
  a.rcinv = static_cast<float>(1.0 / static_cast<double>(p.rc));
  a.H = p.H_fene;
  a.R0 = p.R0;
  a.inv_R0sq = static_cast<float>(1.0 / (static_cast<double>(p.R0) * p.R0));
  a.dt = p.dt;
  a.hdt_m = static_cast<float>(0.5 * static_cast<double>(p.dt) / p.mass);
  a.mass = p.mass;
  a.lambda_star = static_cast<float>(p.lambda_star);
  a.out_scale = p.alpha / p.lambda_star;
  a.seed_lo = static_cast<unsigned>(p.seed & 0xffffffffu);
  a.seed_hi = static_cast<unsigned>(p.seed >> 32);
  a.flow = p.flow_mode;
  a.dpd_on_bonded = p.dpd_on_bonded;
  a.n_rows = p.dim == 2 ? 2 : 5;
  a.excl = std::max(p.exclude_bonds, p.dpd_on_bonded ? 0 : 1);
  a.afbc_peculiar = p.afbc_mode == 1;
  a.chain_len = h->chain_len > 0 ? h->chain_len : 1;
  a.max_beads = h->max_beads;
  a.max_cells = h->max_cells;
  a.n_boxes = h->n_boxes;
  a.id_base = h->id_base;
  a.gm = h->gm;
  a.gm_stride = h->gm_stride;
  a.count_lo = -1;
  a.count_hi = INT_MAX;
  return a;
}

// Launch every size class on its own stream, forked from and joined back
// into `s` with events (capturable into a CUDA graph).
cudaError_t launch_classes(lhmm_micro_s* h, MicroArgs a, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaEventRecord(h->fork, s)) != cudaSuccess) return e;
  for (auto& c : h->classes) {
    if ((e = cudaStreamWaitEvent(c.stream, h->fork, 0)) != cudaSuccess) return e;
    a.list = c.boxes_d;
    a.max_beads = c.max_beads;
    a.max_cells = c.max_cells;
    if ((e = launch_variant(c.variant, a, static_cast<int>(c.boxes.size()),
                            class_smem(c.max_beads, c.max_cells, c.variant), c.stream)) != cudaSuccess)
      return e;
    if ((e = cudaEventRecord(c.done, c.stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, c.done, 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Every box in one persistent launch: a grid of the variant's resident blocks
// on every SM pulls box ids, largest box first, from a device counter.
cudaError_t launch_all_persistent(lhmm_micro_s* h, MicroArgs a, cudaStream_t s) {
  int dev = 0, n_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int v = h->all_variant;
  a.list = h->order_d;
  a.max_beads = h->max_beads;
  a.max_cells = h->max_cells;
  a.work_counter = h->work_counter;
  a.n_items_dev = h->n_all_d;
  a.max_items = h->n_boxes;
  const int grid = std::min(h->n_boxes, kVariants[v].min_blocks * n_sm);
  if ((e = cudaMemsetAsync(h->work_counter, 0, sizeof(int), s)) != cudaSuccess) return e;
  return launch_variant(v, a, grid, class_smem(h->max_beads, h->max_cells, v), s);
}

cudaError_t launch_list(lhmm_micro_s* h, MicroArgs a, const int* list, int v, int grid,
                        cudaStream_t s) {
  a.list = list;
  a.max_beads = h->max_beads;
  a.max_cells = h->max_cells;
  return launch_variant(v, a, grid, class_smem(h->max_beads, h->max_cells, v), s);
}

int sm_count() {
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  return n_sm > 0 ? n_sm : 1;
}

// A list of n boxes known on the host: the latency shape while every box
// can have a resident slot of its own, else the throughput shape.
cudaError_t launch_subset(lhmm_micro_s* h, MicroArgs a, const int* list, int n, cudaStream_t s) {
  const int slots = kVariants[h->subset_variant].min_blocks * sm_count();
  return launch_list(h, a, list, n <= slots ? h->subset_variant : h->list_tp_variant, n, s);
}

}  // namespace

extern "C" lhmm_status lhmm_micro_create(const lhmm_dpd_params* params,
                                         const lhmm_batch_desc* batch, const double* pos0_host,
                                         const float* vel0_host, const float* L0_host,
                                         void* stream, lhmm_micro_t* out) {
  if (!params || !batch || !out || batch->n_boxes < 0) return LHMM_ERR_ARG;
  *out = nullptr;
  const lhmm_dpd_params& p = *params;
  if (!(p.rc > 0.f) || !(p.dt > 0.f) || !(p.mass > 0.f) || !(p.R0 > 0.f) ||
      !(p.lambda_star != 0.0) || p.flow_mode < 0 || p.flow_mode > 2 ||
      (p.dim != 0 && p.dim != 2 && p.dim != 3) || p.exclude_bonds < 0 || p.exclude_bonds > 3 ||
      (p.afbc_mode != 0 && p.afbc_mode != 1))
    return LHMM_ERR_ARG;
  const bool planar = p.dim == 2;
  const int nb = batch->n_boxes;
  if (batch->box_id_offset < 0) return LHMM_ERR_ARG;
  if (nb > 0 && (!batch->box_edge || !batch->n_beads || !batch->n_chains)) return LHMM_ERR_ARG;
  std::vector<BoxInfo> info(nb);
  long long total = 0;
  int max_beads = 1, max_cells = 1;
  for (int b = 0; b < nb; ++b) {
    BoxInfo& B = info[b];
    const int n = batch->n_beads[b], nch = batch->n_chains[b];
    if (n < 0 || n > 65535 || nch < 0) return LHMM_ERR_ARG;
    if (nch > 0 && (batch->chain_len < 2 || (long long)nch * batch->chain_len > n))
      return LHMM_ERR_ARG;
    B.off = total;
    B.n = n;
    B.n_poly = nch * (nch > 0 ? batch->chain_len : 0);
    long long ncell = 1;
    float vol = 1.f;
    for (int a = 0; a < 3; ++a) {
      if (a == 2 && planar) {  // one layer of unit depth that nothing leaves
        B.nc[2] = 1;
        B.w[2] = B.winv[2] = B.len[2] = 1.f;
        B.half_core[2] = B.half_bc[2] = 1e30f;
        continue;
      }
      const float E = batch->box_edge[3 * b + a];
      if (!(E >= 3.f * p.rc)) return LHMM_ERR_ARG;
      B.nc[a] = static_cast<int>(std::floor(E / p.rc));
      B.w[a] = E / static_cast<float>(B.nc[a]);
      B.winv[a] = 1.f / B.w[a];
      B.len[a] = static_cast<float>(B.nc[a]) * B.w[a];
      B.half_core[a] = 0.5f * p.afbc_core_frac * B.len[a];
      B.half_bc[a] = (0.5f * p.afbc_core_frac + p.afbc_bc_frac) * B.len[a];
      ncell *= B.nc[a];
      vol *= (p.flow_mode == LHMM_FLOW_AFBC) ? p.afbc_core_frac * B.len[a] : B.len[a];
    }
    if (ncell > 65535) return LHMM_ERR_UNSUPPORTED;
    // Lees-Edwards rows store the x cell offset of a sliding image in 8 bits
    if (p.flow_mode == LHMM_FLOW_LEES_EDWARDS && B.nc[0] > 60) return LHMM_ERR_UNSUPPORTED;
    B.ncell = static_cast<int>(ncell);
    B.inv_vcore = 1.f / vol;
    total += n;
    max_beads = std::max(max_beads, n);
    max_cells = std::max(max_cells, B.ncell);
  }
  if (total > 0 && (!pos0_host || !vel0_host)) return LHMM_ERR_ARG;
  // queue entries hold 16-bit bead ids (n <= 65535 above); a box too large
  // for one SM's shared memory runs in a global-memory variant
  const size_t optin = max_optin_smem();
  lhmm_micro_s* h = new lhmm_micro_s();
  h->p = p;
  h->n_boxes = nb;
  h->id_base = batch->box_id_offset;
  h->chain_len = batch->chain_len;
  h->max_beads = max_beads;
  h->max_cells = max_cells;
  h->total = total;
  h->info = info;
  h->stream = static_cast<cudaStream_t>(stream);
  h->subset_variant = list_variant(max_beads, max_cells, optin);
  h->list_tp_variant = list_tp_variant(max_beads, max_cells, optin, h->subset_variant);
  auto fail = [&](lhmm_status s) {
    free_micro(h);
    return s;
  };
  if (class_smem(max_beads, max_cells, h->subset_variant) > optin) return fail(LHMM_ERR_UNSUPPORTED);
  // size classes: one per distinct bead count, merged down to at most 12
  std::vector<int> order(nb);
  for (int b = 0; b < nb; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return info[x].n > info[y].n; });  // longest first
  {
    std::vector<std::vector<int>> groups;
    for (int b : order) {
      if (groups.empty() || info[groups.back().front()].n != info[b].n) groups.push_back({});
      groups.back().push_back(b);
    }
    while (groups.size() > 12) {  // merge the two smallest adjacent groups
      size_t best = 0;
      for (size_t g = 1; g + 1 < groups.size(); ++g)
        if (groups[g].size() + groups[g + 1].size() <
            groups[best].size() + groups[best + 1].size())
          best = g;
      groups[best].insert(groups[best].end(), groups[best + 1].begin(), groups[best + 1].end());
      groups.erase(groups.begin() + best + 1);
    }
    for (auto& g : groups) {
      SizeClass c;
      c.boxes = g;
      for (int b : g) {
        c.max_beads = std::max(c.max_beads, info[b].n);
        c.max_cells = std::max(c.max_cells, info[b].ncell);
      }
      c.variant = default_variant(c.max_beads);
      if (class_smem(c.max_beads, c.max_cells, c.variant) > optin) c.variant = 0;
      if (class_smem(c.max_beads, c.max_cells, c.variant) > optin) c.variant = kFirstGmVariant;
      h->classes.push_back(std::move(c));
    }
  }
  const size_t nbx = static_cast<size_t>(std::max(nb, 1));
  const size_t nbead = static_cast<size_t>(std::max(total, 1LL));
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&h->info_d, sizeof(BoxInfo) * nbx)) != cudaSuccess ||
      (e = cudaMalloc(&h->state_d, sizeof(BoxState) * nbx)) != cudaSuccess ||
      (e = cudaMalloc(&h->pos_d, sizeof(float4) * nbead)) != cudaSuccess ||
      (e = cudaMalloc(&h->vel_d, sizeof(float4) * nbead)) != cudaSuccess ||
      (e = cudaMalloc(&h->frc_d, sizeof(float4) * nbead)) != cudaSuccess ||
      (e = cudaMalloc(&h->order_d, sizeof(int) * nbx)) != cudaSuccess ||
      (e = cudaMalloc(&h->L_stage, sizeof(float) * 9 * nbx)) != cudaSuccess ||
      (e = cudaMalloc(&h->st_stage, sizeof(double) * 6 * nbx)) != cudaSuccess ||
      (e = cudaMalloc(&h->sq_stage, sizeof(double) * 6 * nbx)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaMalloc(&h->work_counter, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&h->n_all_d, sizeof(int))) != cudaSuccess ||
      (e = cudaMemcpy(h->n_all_d, &nb, sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(lhmm_cuda_error(e));
  if (kVariants[h->subset_variant].gm && (e = ensure_gm(h)) != cudaSuccess)
    return fail(lhmm_cuda_error(e));
  for (auto& c : h->classes) {
    if ((e = cudaMalloc(&c.boxes_d, sizeof(int) * c.boxes.size())) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMemcpy(c.boxes_d, c.boxes.data(), sizeof(int) * c.boxes.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(lhmm_cuda_error(e));
  }
  // host-side conversion of the initial state to cell-relative form
  std::vector<float4> pos(nbead), vel(nbead), zero(nbead, make_float4(0.f, 0.f, 0.f, 0.f));
  for (int b = 0; b < nb; ++b) {
    const BoxInfo& B = info[b];
    abs_to_rel(B, pos0_host + 3 * B.off, pos.data() + B.off, B.n);
    for (int i = 0; i < B.n; ++i) {
      const float* v = vel0_host + 3 * (B.off + i);
      vel[B.off + i] = make_float4(v[0], v[1], planar ? 0.f : v[2], 0.f);
      if (planar) pos[B.off + i].z = 0.f;
    }
  }
  std::vector<BoxState> st(nbx);
  for (auto& x : st) x = BoxState{0ull, 0.f, 0u};
  cudaStream_t s = h->stream;
  if ((e = cudaMemcpyAsync(h->info_d, info.data(), sizeof(BoxInfo) * nb, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->state_d, st.data(), sizeof(BoxState) * nbx, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->pos_d, pos.data(), sizeof(float4) * total, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->vel_d, vel.data(), sizeof(float4) * total, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->frc_d, zero.data(), sizeof(float4) * total, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->order_d, order.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->L_stage, 0, sizeof(float) * 9 * nbx, s)) != cudaSuccess)
    return fail(lhmm_cuda_error(e));
  if (L0_host && nb > 0 &&
      (e = cudaMemcpyAsync(h->L_stage, L0_host, sizeof(float) * 9 * nb, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
    return fail(lhmm_cuda_error(e));
  // initial forces F(0) from (r0, v0) with the step-0 random stream
  MicroArgs a = make_args(h);
  a.L = h->L_stage;
  a.init_forces = 1;
  a.n_steps = 0;
  if ((e = launch_subset(h, a, h->order_d, nb, s)) != cudaSuccess) return fail(lhmm_cuda_error(e));
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(lhmm_cuda_error(e));
  *out = h;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_micro_destroy(lhmm_micro_t h) {
  if (!h) return LHMM_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  cudaDeviceSynchronize();
  free_micro(h);
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_micro_advance(lhmm_micro_t h, const float* L_dev,
                                          const int* box_idx_dev, int n_active, int n_steps,
                                          double* stress_dev, double* stress_sq_dev,
                                          void* stream) {
  if (!h || n_steps < 0 || n_active < 0) return LHMM_ERR_ARG;
  if (box_idx_dev == nullptr && n_active != h->n_boxes) return LHMM_ERR_ARG;
  if (box_idx_dev != nullptr && n_active > h->n_boxes) return LHMM_ERR_ARG;
  if (n_steps == 0 || n_active == 0) return LHMM_OK;
  if (!L_dev || !stress_dev) return LHMM_ERR_ARG;
  MicroArgs a = make_args(h);
  a.L = L_dev;
  a.stress = stress_dev;
  a.stress_sq = stress_sq_dev;
  a.n_steps = n_steps;
  a.init_forces = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (box_idx_dev) {
    LHMM_CK(launch_subset(h, a, box_idx_dev, n_active, s));
  } else if (h->all_persistent) {
    LHMM_CK(launch_all_persistent(h, a, s));
  } else {
    LHMM_CK(launch_classes(h, a, s));
  }
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_micro_advance_dev_count(lhmm_micro_t h, const float* L_dev,
                                                    const int* box_idx_dev,
                                                    const int* n_active_dev, int max_active,
                                                    int n_steps, double* stress_dev,
                                                    double* stress_sq_dev, void* stream) {
  if (!h || !box_idx_dev || !n_active_dev || max_active < 0 || n_steps < 0) return LHMM_ERR_ARG;
  if (max_active > h->n_boxes) return LHMM_ERR_ARG;
  if (n_steps == 0 || max_active == 0) return LHMM_OK;
  if (!L_dev || !stress_dev) return LHMM_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MicroArgs a = make_args(h);
  a.L = L_dev;
  a.stress = stress_dev;
  a.stress_sq = stress_sq_dev;
  a.n_steps = n_steps;
  a.init_forces = 0;
  a.work_counter = h->work_counter;
  a.n_items_dev = n_active_dev;
  a.max_items = max_active;
  const int n_sm = sm_count();
  // The item count is known only on the device, so two persistent launches
  // are queued and each leaves the items to the other outside its range:
  // up to one box per resident slot of the latency shape (each box on an SM
  // of its own), the throughput shape beyond.
  const int lat = h->subset_variant, tp = h->list_tp_variant;
  const int slots = kVariants[lat].min_blocks * n_sm;
  LHMM_CK(cudaMemsetAsync(h->work_counter, 0, sizeof(int), s));
  if (lat == tp || max_active <= slots) {
    LHMM_CK(launch_list(h, a, box_idx_dev, lat,
                        std::min(max_active, kVariants[lat].min_blocks * n_sm), s));
    return LHMM_OK;
  }
  a.count_hi = slots;
  LHMM_CK(launch_list(h, a, box_idx_dev, lat, slots, s));
  a.count_lo = slots;
  a.count_hi = INT_MAX;
  LHMM_CK(launch_list(h, a, box_idx_dev, tp,
                      std::min(max_active, kVariants[tp].min_blocks * n_sm), s));
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_micro_diagnostics(lhmm_micro_t h, double* diag_dev, void* stream) {
  if (!h || !diag_dev) return LHMM_ERR_ARG;
  if (h->n_boxes == 0) return LHMM_OK;
  MicroArgs a = make_args(h);
  micro_diagnostics_kernel<<<h->n_boxes, kDiagThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      a, diag_dev);
  LHMM_CK(cudaGetLastError());
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_micro_advance_host(lhmm_micro_t h, const float* L_host, int n_steps,
                                               double* stress_host, double* stress_sq_host,
                                               void* stream) {
  if (!h || !L_host || !stress_host || n_steps < 0) return LHMM_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nb = static_cast<size_t>(h->n_boxes);
  LHMM_CK(cudaMemcpyAsync(h->L_stage, L_host, sizeof(float) * 9 * nb, cudaMemcpyHostToDevice, s));
  lhmm_status st = lhmm_micro_advance(h, h->L_stage, nullptr, h->n_boxes, n_steps, h->st_stage,
                                      stress_sq_host ? h->sq_stage : nullptr, stream);
  if (st != LHMM_OK) return st;
  LHMM_CK(cudaMemcpyAsync(stress_host, h->st_stage, sizeof(double) * 6 * nb, cudaMemcpyDeviceToHost, s));
  if (stress_sq_host)
    LHMM_CK(cudaMemcpyAsync(stress_sq_host, h->sq_stage, sizeof(double) * 6 * nb,
                            cudaMemcpyDeviceToHost, s));
  LHMM_CK(cudaStreamSynchronize(s));
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_micro_sync(lhmm_micro_t h, uint32_t* box_status_host) {
  if (!h) return LHMM_ERR_ARG;
  LHMM_CK(cudaDeviceSynchronize());
  std::vector<BoxState> st(static_cast<size_t>(std::max(h->n_boxes, 1)));
  LHMM_CK(cudaMemcpy(st.data(), h->state_d, sizeof(BoxState) * h->n_boxes, cudaMemcpyDeviceToHost));
  unsigned all = 0;
  for (int b = 0; b < h->n_boxes; ++b) {
    if (box_status_host) box_status_host[b] = st[b].status;
    all |= st[b].status;
    st[b].status = 0;
  }
  if (all) LHMM_CK(cudaMemcpy(h->state_d, st.data(), sizeof(BoxState) * h->n_boxes, cudaMemcpyHostToDevice));
  if (all & LHMM_BOX_BOND_OVERSTRETCH) return LHMM_ERR_BOND_OVERSTRETCH;
  if (all & LHMM_BOX_NAN) return LHMM_ERR_NAN;
  if (all & LHMM_BOX_CELL_OVERFLOW) return LHMM_ERR_CELL_OVERFLOW;
  if (all & LHMM_BOX_FORCE_RANGE) return LHMM_ERR_FORCE_RANGE;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_micro_get_state(lhmm_micro_t h, int box, double* pos_host,
                                            float* vel_host, float* force_host, uint64_t* step,
                                            float* le_offset) {
  if (!h || box < 0 || box >= h->n_boxes) return LHMM_ERR_ARG;
  LHMM_CK(cudaStreamSynchronize(h->stream));
  LHMM_CK(cudaDeviceSynchronize());
  const BoxInfo& B = h->info[box];
  std::vector<float4> buf(static_cast<size_t>(std::max(B.n, 1)));
  if (pos_host && B.n) {
    LHMM_CK(cudaMemcpy(buf.data(), h->pos_d + B.off, sizeof(float4) * B.n, cudaMemcpyDeviceToHost));
    rel_to_abs(B, buf.data(), pos_host, B.n);
  }
  float* outs[2] = {vel_host, force_host};
  float4* srcs[2] = {h->vel_d, h->frc_d};
  for (int k = 0; k < 2; ++k) {
    if (!outs[k] || !B.n) continue;
    LHMM_CK(cudaMemcpy(buf.data(), srcs[k] + B.off, sizeof(float4) * B.n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < B.n; ++i) {
      outs[k][3 * i] = buf[i].x;
      outs[k][3 * i + 1] = buf[i].y;
      outs[k][3 * i + 2] = buf[i].z;
    }
  }
  if (step || le_offset) {
    BoxState s;
    LHMM_CK(cudaMemcpy(&s, h->state_d + box, sizeof(BoxState), cudaMemcpyDeviceToHost));
    if (step) *step = s.step;
    if (le_offset) *le_offset = s.le_offset;
  }
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_micro_set_state(lhmm_micro_t h, int box, const double* pos_host,
                                            const float* vel_host, const float* force_host,
                                            uint64_t step, float le_offset) {
  if (!h || box < 0 || box >= h->n_boxes || !pos_host || !vel_host || !force_host)
    return LHMM_ERR_ARG;
  LHMM_CK(cudaDeviceSynchronize());
  const BoxInfo& B = h->info[box];
  if (B.n) {
    std::vector<float4> buf(static_cast<size_t>(B.n));
    const bool planar = h->p.dim == 2;  // z components are zero in 2D
    abs_to_rel(B, pos_host, buf.data(), B.n);
    if (planar)
      for (int i = 0; i < B.n; ++i) buf[i].z = 0.f;
    LHMM_CK(cudaMemcpy(h->pos_d + B.off, buf.data(), sizeof(float4) * B.n, cudaMemcpyHostToDevice));
    for (int i = 0; i < B.n; ++i)
      buf[i] = make_float4(vel_host[3 * i], vel_host[3 * i + 1], planar ? 0.f : vel_host[3 * i + 2], 0.f);
    LHMM_CK(cudaMemcpy(h->vel_d + B.off, buf.data(), sizeof(float4) * B.n, cudaMemcpyHostToDevice));
    for (int i = 0; i < B.n; ++i)
      buf[i] = make_float4(force_host[3 * i], force_host[3 * i + 1], planar ? 0.f : force_host[3 * i + 2], 0.f);
    LHMM_CK(cudaMemcpy(h->frc_d + B.off, buf.data(), sizeof(float4) * B.n, cudaMemcpyHostToDevice));
  }
  BoxState s{step, le_offset, 0u};
  LHMM_CK(cudaMemcpy(h->state_d + box, &s, sizeof(BoxState), cudaMemcpyHostToDevice));
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_micro_info(lhmm_micro_t h, int* n_boxes, int64_t* total_beads,
                                       int* max_beads) {
  if (!h) return LHMM_ERR_ARG;
  if (n_boxes) *n_boxes = h->n_boxes;
  if (total_beads) *total_beads = h->total;
  if (max_beads) *max_beads = h->max_beads;
  return LHMM_OK;
}

namespace {
// process-wide autotune cache: (largest box, cells, flow, device) -> variant
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune_cache;
}  // namespace

extern "C" lhmm_status lhmm_micro_autotune(lhmm_micro_t h, const float* L_dev, int probe_steps,
                                           void* stream) {
  if (!h || !L_dev || probe_steps < 1) return LHMM_ERR_ARG;
  if (h->total == 0) return LHMM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  LHMM_CK(cudaGetDevice(&dev));
  LHMM_CK(cudaStreamSynchronize(s));
  LHMM_CK(cudaDeviceSynchronize());
  const size_t nb = static_cast<size_t>(h->n_boxes), nt = static_cast<size_t>(h->total);
  float4 *sp = nullptr, *sv = nullptr, *sf = nullptr;
  BoxState* ss = nullptr;
  cudaError_t e;
  auto cleanup = [&]() {
    cudaFree(sp);
    cudaFree(sv);
    cudaFree(sf);
    cudaFree(ss);
  };
  if ((e = cudaMalloc(&sp, sizeof(float4) * nt)) != cudaSuccess ||
      (e = cudaMalloc(&sv, sizeof(float4) * nt)) != cudaSuccess ||
      (e = cudaMalloc(&sf, sizeof(float4) * nt)) != cudaSuccess ||
      (e = cudaMalloc(&ss, sizeof(BoxState) * nb)) != cudaSuccess ||
      (e = cudaMemcpy(sp, h->pos_d, sizeof(float4) * nt, cudaMemcpyDeviceToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(sv, h->vel_d, sizeof(float4) * nt, cudaMemcpyDeviceToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(sf, h->frc_d, sizeof(float4) * nt, cudaMemcpyDeviceToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ss, h->state_d, sizeof(BoxState) * nb, cudaMemcpyDeviceToDevice)) != cudaSuccess) {
    cleanup();
    return lhmm_cuda_error(e);
  }
  const size_t optin = max_optin_smem();
  MicroArgs a = make_args(h);
  a.L = L_dev;
  a.stress = h->st_stage;
  a.stress_sq = nullptr;
  a.n_steps = probe_steps;
  a.init_forces = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  lhmm_status result = LHMM_OK;
  int tuned_all = 0;
  for (auto& c : h->classes) {
    const auto key = std::make_tuple(c.max_beads, c.max_cells, h->p.flow_mode, dev);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        c.variant = it->second;
        continue;
      }
    }
    a.list = c.boxes_d;
    a.max_beads = c.max_beads;
    a.max_cells = c.max_cells;
    float best = 1e30f;
    int best_v = c.variant;
    // global-memory variants only for classes no shared-memory variant holds
    const bool big = !fits_shared(c.max_beads, c.max_cells, optin);
    for (int v = 0; v < kNumVariants; ++v) {
      const size_t sm = class_smem(c.max_beads, c.max_cells, v);
      if (sm > optin || kVariants[v].gm != big) continue;
      const int grid = static_cast<int>(c.boxes.size());
      float ms = 0.f;
      if ((e = launch_variant(v, a, grid, sm, s)) != cudaSuccess ||  // warm-up
          (e = cudaEventRecord(e0, s)) != cudaSuccess ||
          (e = launch_variant(v, a, grid, sm, s)) != cudaSuccess ||
          (e = cudaEventRecord(e1, s)) != cudaSuccess ||
          (e = cudaEventSynchronize(e1)) != cudaSuccess ||
          (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
        result = lhmm_cuda_error(e);
        break;
      }
      if (ms < best) {
        best = ms;
        best_v = v;
      }
    }
    if (result != LHMM_OK) break;
    c.variant = best_v;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best_v;
  }
  // the whole batch: the tuned class plan against one persistent launch over
  // every box (largest first) in each variant that holds the largest box
  h->all_persistent = false;
  if (result == LHMM_OK && h->classes.size() > 1) {
    auto time_it = [&](auto launch, float& ms) -> cudaError_t {
      cudaError_t x;
      if ((x = launch()) != cudaSuccess || (x = cudaEventRecord(e0, s)) != cudaSuccess ||
          (x = launch()) != cudaSuccess || (x = cudaEventRecord(e1, s)) != cudaSuccess ||
          (x = cudaEventSynchronize(e1)) != cudaSuccess)
        return x;
      return cudaEventElapsedTime(&ms, e0, e1);
    };
    float best = 1e30f;
    e = time_it([&]() { return launch_classes(h, a, s); }, best);
    const bool big = !fits_shared(h->max_beads, h->max_cells, optin);
    for (int v = 0; v < kNumVariants && e == cudaSuccess; ++v) {
      if (class_smem(h->max_beads, h->max_cells, v) > optin || kVariants[v].gm != big) continue;
      if (kVariants[v].gm && (e = ensure_gm(h)) != cudaSuccess) break;
      h->all_variant = v;
      float ms = 0.f;
      if ((e = time_it([&]() { return launch_all_persistent(h, a, s); }, ms)) != cudaSuccess) break;
      if (ms < best) {
        best = ms;
        h->all_persistent = true;
        tuned_all = v;
      }
    }
    if (e != cudaSuccess) {
      result = lhmm_cuda_error(e);
      h->all_persistent = false;
    }
    if (h->all_persistent) h->all_variant = tuned_all;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore the state the probes advanced
  if ((e = cudaMemcpy(h->pos_d, sp, sizeof(float4) * nt, cudaMemcpyDeviceToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(h->vel_d, sv, sizeof(float4) * nt, cudaMemcpyDeviceToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(h->frc_d, sf, sizeof(float4) * nt, cudaMemcpyDeviceToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(h->state_d, ss, sizeof(BoxState) * nb, cudaMemcpyDeviceToDevice)) != cudaSuccess) {
    cleanup();
    return lhmm_cuda_error(e);
  }
  cleanup();
  return result;
}

extern "C" lhmm_status lhmm_micro_plan(lhmm_micro_t h, int* n_classes, int cap, int* class_boxes,
                                       int* class_max_beads, int* class_threads,
                                       int* class_min_blocks) {
  if (!h || !n_classes) return LHMM_ERR_ARG;
  if (h->all_persistent) {  // one launch over every box
    *n_classes = 1;
    if (cap > 0) {
      if (class_boxes) class_boxes[0] = h->n_boxes;
      if (class_max_beads) class_max_beads[0] = h->max_beads;
      if (class_threads) class_threads[0] = kVariants[h->all_variant].threads;
      if (class_min_blocks) class_min_blocks[0] = kVariants[h->all_variant].min_blocks;
    }
    return LHMM_OK;
  }
  *n_classes = static_cast<int>(h->classes.size());
  for (int k = 0; k < cap && k < *n_classes; ++k) {
    const SizeClass& c = h->classes[k];
    if (class_boxes) class_boxes[k] = static_cast<int>(c.boxes.size());
    if (class_max_beads) class_max_beads[k] = c.max_beads;
    if (class_threads) class_threads[k] = kVariants[c.variant].threads;
    if (class_min_blocks) class_min_blocks[k] = kVariants[c.variant].min_blocks;
  }
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_micro_set_list_variant(lhmm_micro_t h, int variant) {
  if (!h || variant < -1 || variant >= kNumVariants) return LHMM_ERR_ARG;
  const size_t optin = max_optin_smem();
  int v = variant, tp = variant;
  if (variant < 0) {
    v = list_variant(h->max_beads, h->max_cells, optin);
    tp = list_tp_variant(h->max_beads, h->max_cells, optin, v);
  }
  if (class_smem(h->max_beads, h->max_cells, v) > optin) return LHMM_ERR_UNSUPPORTED;
  if (kVariants[v].gm || kVariants[tp].gm) LHMM_CK(ensure_gm(h));
  h->subset_variant = v;
  h->list_tp_variant = tp;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_micro_set_variant(lhmm_micro_t h, int cls, int variant) {
  if (!h || variant < 0 || variant >= kNumVariants) return LHMM_ERR_ARG;
  if (cls < 0 || cls >= static_cast<int>(h->classes.size())) return LHMM_ERR_ARG;
  SizeClass& c = h->classes[cls];
  if (class_smem(c.max_beads, c.max_cells, variant) > max_optin_smem()) return LHMM_ERR_UNSUPPORTED;
  if (kVariants[variant].gm) LHMM_CK(ensure_gm(h));
  c.variant = variant;
  h->all_persistent = false;  // an explicit class variant means the class plan
  return LHMM_OK;
}
