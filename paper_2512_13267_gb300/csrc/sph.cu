// sph.cu -- macroscale SPH of the LHMM (arXiv 2512.13267, Sec. 3.2: Eqs.
// sph_continuity and tait; Sec. 3.4: Eq. macro_micro) on sm_103a.
//
// 2D weakly compressible SPH in a periodic box.  Per substep: half kick and
// drift (velocity-Verlet, coupling protocol Step 1), a counting-sort cell
// list with cells >= h wide and ascending particle order inside each cell,
// summation number density d_I = sum_J W_IJ (self included) with the Tait
// pressure, and the momentum sum: pressure, Espanol-Revenga viscous pair
// term with the half-step velocity, and the micro-stress coupling term
// -(pi_I/d_I^2 + pi_J/d_J^2) F_IJ r_IJ, plus the body force; then the second
// half kick.  After the substeps the velocity gradient of every fluid
// particle, L_ab = dv_a/dx_b = sum_J (F_IJ/d_J) v_IJ,a r_IJ,b, is exported as
// a 3x3 tensor for its micro-domain.  A group of 8 or 16 lanes shares one
// particle: each lane takes every 8th or 16th slot of the 3x3 neighbour
// cells, row by row in a fixed order, and the group adds its partial sums
// with a fixed butterfly, so a step is bit-reproducible.  A substep is four launches:
// kicks, drift and binning in one pass (the previous substep's closing half
// kick folded in), the cell list (one block for systems of up to 8192
// particles and cells, else scan, scatter and in-cell sort), the density
// with the per-particle factors of the momentum sum (p/d^2 and pi/d^2), and
// the forces.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include "lhmm_common.cuh"

namespace {

struct SphArgs {
  int n, n_fluid, ncx, ncy, ncell;
  float Lx, Ly, cwx, cwy, h, hinv, mass, rho0, c2rho0_7, pb, a_visc, b_visc, dt;
  int kernel, body_mode;
  float bfx, bfy;
  float2 *pos, *vel, *acc;
  float *d, *p;
  const int* wall;
  int *cnt, *start, *perm, *cell_of;
  // per-particle factors of the momentum sum, written with the density:
  // p/d^2 and the micro stress over d^2 (xx, xy, yy; zero where a particle
  // carries none).  NULL where only densities and gradients are wanted.
  float* pterm;
  float4* sterm;
};

__device__ __forceinline__ float kernel_W(int kind, float r, float h, float hinv) {
  const float q = r * hinv;
  if (q >= 1.f) return 0.f;
  const float omq = 1.f - q;
  const float inv_h2_pi = hinv * hinv * 0.318309886183790672f;  // 1/(pi h^2)
  if (kind == LHMM_SPH_LUCY) return 5.f * inv_h2_pi * (1.f + 3.f * q) * omq * omq * omq;
  return 7.f * inv_h2_pi * (1.f + 4.f * q) * omq * omq * omq * omq;
}

// F(r) = -W'(r)/r
__device__ __forceinline__ float kernel_F(int kind, float r, float hinv) {
  const float q = r * hinv;
  if (q >= 1.f) return 0.f;
  const float omq = 1.f - q;
  const float h4 = hinv * hinv * hinv * hinv * 0.318309886183790672f;
  if (kind == LHMM_SPH_LUCY) return 60.f * h4 * omq * omq;
  return 140.f * h4 * omq * omq * omq;
}

__device__ __forceinline__ float2 min_image(float2 a, float2 b, float Lx, float Ly) {
  float dx = a.x - b.x, dy = a.y - b.y;
  dx -= Lx * rintf(dx / Lx);
  dy -= Ly * rintf(dy / Ly);
  return make_float2(dx, dy);
}

// Cell of a position, taken at its periodic image in [0, L): positions the
// caller passes outside the box (the allocation-free entry point takes them
// as given) bin where their image lies; inside the box the wrap is exact (it
// subtracts zero), so in-box positions bin as before.
__device__ __forceinline__ int cell_index(float2 r, const SphArgs& A) {
  const float x = r.x - A.Lx * floorf(r.x / A.Lx), y = r.y - A.Ly * floorf(r.y / A.Ly);
  int cx = static_cast<int>(floorf(x / A.cwx)), cy = static_cast<int>(floorf(y / A.cwy));
  cx = min(max(cx, 0), A.ncx - 1);
  cy = min(max(cy, 0), A.ncy - 1);
  return cx + A.ncx * cy;
}

__global__ void sph_kick_drift(SphArgs A, float half_dt, int drift) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= A.n || A.wall[I]) return;
  float2 v = A.vel[I];
  const float2 a = A.acc[I];
  v.x += half_dt * a.x;
  v.y += half_dt * a.y;
  A.vel[I] = v;
  if (drift) {
    float2 r = A.pos[I];
    r.x += A.dt * v.x;
    r.y += A.dt * v.y;
    r.x -= A.Lx * floorf(r.x / A.Lx);
    r.y -= A.Ly * floorf(r.y / A.Ly);
    if (r.x >= A.Lx) r.x -= A.Lx;
    if (r.y >= A.Ly) r.y -= A.Ly;
    A.pos[I] = r;
  }
}

// The start of a substep in one pass: n_kicks half kicks with the current
// acceleration (two when the previous substep's closing half kick is folded
// in; the same two additions, in the same order, as two separate passes),
// the drift, then the particle's cell and its count for the cell list.
__global__ void sph_kick_drift_bin(SphArgs A, float half_dt, int n_kicks, int drift) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= A.n) return;
  float2 r = A.pos[I];
  if (!A.wall[I] && (n_kicks > 0 || drift)) {
    float2 v = A.vel[I];
    const float2 a = A.acc[I];
    for (int k = 0; k < n_kicks; ++k) {
      v.x += half_dt * a.x;
      v.y += half_dt * a.y;
    }
    A.vel[I] = v;
    if (drift) {
      r.x += A.dt * v.x;
      r.y += A.dt * v.y;
      r.x -= A.Lx * floorf(r.x / A.Lx);
      r.y -= A.Ly * floorf(r.y / A.Ly);
      if (r.x >= A.Lx) r.x -= A.Lx;
      if (r.y >= A.Ly) r.y -= A.Ly;
      A.pos[I] = r;
    }
  }
  const int c = cell_index(r, A);
  A.cell_of[I] = c;
  atomicAdd(&A.cnt[c], 1);
}

// Counting sort by cell in four launches: bin and count (cnt must be zero on
// entry), exclusive scan in one block (which clears cnt for use as cursors),
// scatter, and an ascending-index sort inside each cell, which leaves cnt zero
// again for the next build.
__global__ void sph_bin(SphArgs A) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= A.n) return;
  const int c = cell_index(A.pos[I], A);
  A.cell_of[I] = c;
  atomicAdd(&A.cnt[c], 1);
}

// exclusive scan of the cell counts into start (one block; clears cnt)
__device__ __forceinline__ void scan_counts(const SphArgs& A) {
  __shared__ int warp_tot[32];
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int per = (A.ncell + T - 1) / T;
  const int c0 = min(tid * per, A.ncell), c1 = min(c0 + per, A.ncell);
  int local = 0;
  for (int c = c0; c < c1; ++c) local += A.cnt[c];
  int x = local;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = T / 32;
    int y = lane < nw ? warp_tot[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    if (lane < nw) warp_tot[lane] = y;
  }
  __syncthreads();
  int run = (warp > 0 ? warp_tot[warp - 1] : 0) + x - local;
  for (int c = c0; c < c1; ++c) {
    A.start[c] = run;
    run += A.cnt[c];
    A.cnt[c] = 0;
  }
  if (tid == 0) A.start[A.ncell] = A.n;
}

__global__ void sph_scan(SphArgs A) { scan_counts(A); }

__global__ void sph_scatter(SphArgs A) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= A.n) return;
  const int c = A.cell_of[I];
  A.perm[A.start[c] + atomicAdd(&A.cnt[c], 1)] = I;
}

// One warp per cell: a cell of up to 32 particles is ranked with shuffles
// (rank = number of smaller indices) and written back in ascending order;
// larger cells (far denser than any SPH state) fall back to an insertion
// sort by lane 0.
__device__ __forceinline__ void sort_cell(const SphArgs& A, int c, int lane) {
  const int s0 = A.start[c], m = A.start[c + 1] - s0;
  if (m <= 32) {
    const int key = lane < m ? A.perm[s0 + lane] : 0x7fffffff;
    int rank = 0;
    for (int t = 0; t < m; ++t) rank += __shfl_sync(0xffffffffu, key, t) < key;
    __syncwarp();
    if (lane < m) A.perm[s0 + rank] = key;
  } else if (lane == 0) {
    for (int q = s0 + 1; q < s0 + m; ++q) {
      const int key = A.perm[q];
      int k = q - 1;
      while (k >= s0 && A.perm[k] > key) {
        A.perm[k + 1] = A.perm[k];
        --k;
      }
      A.perm[k + 1] = key;
    }
  }
  if (lane == 0) A.cnt[c] = 0;
}

__global__ void sph_cellsort(SphArgs A) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (c >= A.ncell) return;  // whole warp
  sort_cell(A, c, lane);
}

// The start of a substep of a small system in one block, with the cell
// list built in shared memory: the half kicks and drift of
// sph_kick_drift_bin (same arithmetic), then count, exclusive scan, scatter
// and in-cell sort by particle index, the same cell list as the launches
// above; start and perm are copied out for the neighbour sums, and the
// global counters are not touched (they stay zero).
__global__ void __launch_bounds__(1024) sph_substep_cells_block(SphArgs A, float half_dt,
                                                                int n_kicks, int drift) {
  extern __shared__ int sm[];
  int* cnt = sm;                      // ncell counters, then cursors
  int* start = cnt + A.ncell;         // ncell + 1 cell starts
  int* perm = start + A.ncell + 1;    // n slots
  __shared__ int warp_tot[32];
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  for (int c = tid; c < A.ncell; c += T) cnt[c] = 0;
  __syncthreads();
  for (int I = tid; I < A.n; I += T) {
    float2 r = A.pos[I];
    if (!A.wall[I] && (n_kicks > 0 || drift)) {
      float2 v = A.vel[I];
      const float2 a = A.acc[I];
      for (int k = 0; k < n_kicks; ++k) {
        v.x += half_dt * a.x;
        v.y += half_dt * a.y;
      }
      A.vel[I] = v;
      if (drift) {
        r.x += A.dt * v.x;
        r.y += A.dt * v.y;
        r.x -= A.Lx * floorf(r.x / A.Lx);
        r.y -= A.Ly * floorf(r.y / A.Ly);
        if (r.x >= A.Lx) r.x -= A.Lx;
        if (r.y >= A.Ly) r.y -= A.Ly;
        A.pos[I] = r;
      }
    }
    const int c = cell_index(r, A);
    A.cell_of[I] = c;
    atomicAdd(&cnt[c], 1);
  }
  __syncthreads();
  // exclusive scan of the counts (each thread a contiguous range of cells)
  const int per = (A.ncell + T - 1) / T;
  const int c0 = min(tid * per, A.ncell), c1 = min(c0 + per, A.ncell);
  int local = 0;
  for (int c = c0; c < c1; ++c) local += cnt[c];
  int x = local;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int y = lane < nw ? warp_tot[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    if (lane < nw) warp_tot[lane] = y;
  }
  __syncthreads();
  int run = (warp > 0 ? warp_tot[warp - 1] : 0) + x - local;
  for (int c = c0; c < c1; ++c) {
    start[c] = run;
    run += cnt[c];
    cnt[c] = 0;
  }
  if (tid == 0) start[A.ncell] = A.n;
  __syncthreads();
  for (int I = tid; I < A.n; I += T) {
    const int c = A.cell_of[I];
    perm[start[c] + atomicAdd(&cnt[c], 1)] = I;
  }
  __syncthreads();
  // ascending particle index inside each cell: one warp per cell
  for (int c = warp; c < A.ncell; c += nw) {
    const int s0 = start[c], m = start[c + 1] - s0;
    if (m <= 32) {
      const int key = lane < m ? perm[s0 + lane] : 0x7fffffff;
      int rank = 0;
      for (int t = 0; t < m; ++t) rank += __shfl_sync(0xffffffffu, key, t) < key;
      __syncwarp();
      if (lane < m) perm[s0 + rank] = key;
    } else if (lane == 0) {
      for (int q = s0 + 1; q < s0 + m; ++q) {
        const int key = perm[q];
        int k = q - 1;
        while (k >= s0 && perm[k] > key) {
          perm[k + 1] = perm[k];
          --k;
        }
        perm[k + 1] = key;
      }
    }
    __syncwarp();
  }
  __syncthreads();
  for (int c = tid; c <= A.ncell; c += T) A.start[c] = start[c];
  for (int q = tid; q < A.n; q += T) A.perm[q] = perm[q];
}

// Scan, scatter and in-cell sort of a small system in one block: the same
// cell list as the three launches above, without the gaps between them.
__global__ void __launch_bounds__(1024) sph_cells_block(SphArgs A) {
  scan_counts(A);
  __syncthreads();
  for (int I = threadIdx.x; I < A.n; I += blockDim.x) {
    const int c = A.cell_of[I];
    A.perm[A.start[c] + atomicAdd(&A.cnt[c], 1)] = I;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = threadIdx.x >> 5; c < A.ncell; c += nw) sort_cell(A, c, lane);
}

// lanes per particle in the neighbour sums: 16 for small systems (more
// parallelism where too few particles keep the SMs busy), 8 above
// kSmallSystem particles (fewer lanes wasted on short slot runs)
constexpr int kSmallSystem = 8192;
constexpr int kTinySystem = 4096;  // a whole warp per particle up to here

// Visits lane g's share of the 3x3 cell neighbourhood of particle I, row by
// row (dy = -1, 0, 1): the three cells x-1, x, x+1 of a row are consecutive
// cell indices, so their particles are one run of cell-list slots (two runs
// where the row wraps around x), and the lane takes every G-th slot of each
// run starting at g.  The order is fixed, so the sums are bit-reproducible.
template <int G, typename F>
__device__ __forceinline__ void for_neighbours(const SphArgs& A, int I, int g, F&& fn) {
  const int c = A.cell_of[I];
  const int cx = c % A.ncx, cy = c / A.ncx;
  for (int dy = -1; dy <= 1; ++dy) {
    int y = cy + dy;
    y += (y < 0) ? A.ncy : 0;
    y -= (y >= A.ncy) ? A.ncy : 0;
    const int row = A.ncx * y;
    // runs [a0, a1) and [b0, b1) of cells; the second is empty without wrap
    int a0 = cx - 1, a1 = cx + 2, b0 = 0, b1 = 0;
    if (cx == 0) {
      a0 = A.ncx - 1; a1 = A.ncx; b0 = 0; b1 = 2;
    } else if (cx == A.ncx - 1) {
      a0 = cx - 1; a1 = A.ncx; b0 = 0; b1 = 1;
    }
    for (int q = A.start[row + a0] + g, e = A.start[row + a1]; q < e; q += G) fn(A.perm[q]);
    for (int q = A.start[row + b0] + g, e = A.start[row + b1]; q < e; q += G) fn(A.perm[q]);
  }
}

// Sum over the G lanes of a group (every lane of the warp takes part;
// a + b == b + a exactly, so every lane of the group gets the same bits).
template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int G>
__global__ void sph_density(SphArgs A, const double* stress) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int I = t / G, g = t % G;
  const bool valid = I < A.n;
  float s = 0.f;
  if (valid) {
    const float2 ri = A.pos[I];
    for_neighbours<G>(A, I, g, [&](int J) {
      const float2 r = min_image(ri, A.pos[J], A.Lx, A.Ly);
      s += kernel_W(A.kernel, sqrtf(r.x * r.x + r.y * r.y), A.h, A.hinv);
    });
  }
  s = group_sum<G>(s);
  if (valid && g == 0) {
    A.d[I] = s;
    const float rr = A.mass * s / A.rho0;
    const float r2 = rr * rr, r4 = r2 * r2;
    const float p = A.c2rho0_7 * (r4 * r2 * rr - 1.f) + A.pb;  // Eq. tait
    A.p[I] = p;
    if (A.pterm) {  // the factors every neighbour's momentum sum reads
      const float inv = 1.f / (s * s);
      A.pterm[I] = p * inv;
      float4 st = make_float4(0.f, 0.f, 0.f, 0.f);
      if (stress && I < A.n_fluid && !A.wall[I]) {
        st.x = static_cast<float>(stress[6 * I + 0]) * inv;
        st.y = static_cast<float>(stress[6 * I + 3]) * inv;
        st.z = static_cast<float>(stress[6 * I + 1]) * inv;
      }
      A.sterm[I] = st;
    }
  }
}

template <int G>
__global__ void sph_force(SphArgs A, const double* stress) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int I = t / G, g = t % G;
  const bool active = I < A.n && !A.wall[I];
  float fx = 0.f, fy = 0.f;
  float2 ri = make_float2(0.f, 0.f);
  if (active) {
    ri = A.pos[I];
    const float2 vi = A.vel[I];
    const float di = A.d[I];
    const float Pi = A.pterm[I];
    float sxx = 0.f, sxy = 0.f, syy = 0.f;
    if (stress) {
      const float4 si = A.sterm[I];
      sxx = si.x;
      sxy = si.y;
      syy = si.z;
    }
    for_neighbours<G>(A, I, g, [&](int J) {
      if (J == I) return;
      const float2 r = min_image(ri, A.pos[J], A.Lx, A.Ly);
      const float rr = sqrtf(r.x * r.x + r.y * r.y);
      const float F = kernel_F(A.kernel, rr, A.hinv);
      if (F == 0.f || rr == 0.f) return;  // e_IJ undefined for coincident particles
      const float dj = A.d[J];
      const float P = Pi + A.pterm[J];
      fx += P * F * r.x;
      fy += P * F * r.y;
      const float2 vj = A.vel[J];
      const float vx = vi.x - vj.x, vy = vi.y - vj.y;
      const float inv_r = 1.f / rr;
      const float ex = r.x * inv_r, ey = r.y * inv_r;
      const float ve = vx * ex + vy * ey;
      const float cv = F / (di * dj);
      fx -= (A.a_visc * vx + A.b_visc * ve * ex) * cv;
      fy -= (A.a_visc * vy + A.b_visc * ve * ey) * cv;
      if (stress) {
        const float4 sj = A.sterm[J];  // zero for wall particles
        const float jxx = sxx + sj.x, jxy = sxy + sj.y, jyy = syy + sj.z;
        fx -= (jxx * r.x + jxy * r.y) * F;
        fy -= (jxy * r.x + jyy * r.y) * F;
      }
    });
  }
  fx = group_sum<G>(fx);
  fy = group_sum<G>(fy);
  if (I < A.n && g == 0) {
    if (!active) {
      A.acc[I] = make_float2(0.f, 0.f);  // wall particles stay fixed
    } else {
      float gx = A.bfx, gy = A.bfy;
      if (A.body_mode == LHMM_SPH_BODY_REVERSE_POISEUILLE) {
        gx = (ri.y >= 0.5f * A.Ly) ? A.bfx : -A.bfx;
        gy = 0.f;
      }
      A.acc[I] = make_float2(fx / A.mass + gx, fy / A.mass + gy);
    }
  }
}

template <int G>
__global__ void sph_velgrad(SphArgs A, float* L_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int I = t / G, g = t % G;
  const bool valid = I < A.n_fluid;
  float Lxx = 0.f, Lxy = 0.f, Lyx = 0.f, Lyy = 0.f;
  if (valid) {
    const float2 ri = A.pos[I], vi = A.vel[I];
    for_neighbours<G>(A, I, g, [&](int J) {
      if (J == I) return;
      const float2 r = min_image(ri, A.pos[J], A.Lx, A.Ly);
      const float F = kernel_F(A.kernel, sqrtf(r.x * r.x + r.y * r.y), A.hinv);
      if (F == 0.f) return;
      const float2 vj = A.vel[J];
      const float cf = F / A.d[J];
      const float vx = vi.x - vj.x, vy = vi.y - vj.y;
      Lxx += cf * vx * r.x;
      Lxy += cf * vx * r.y;
      Lyx += cf * vy * r.x;
      Lyy += cf * vy * r.y;
    });
  }
  Lxx = group_sum<G>(Lxx);
  Lxy = group_sum<G>(Lxy);
  Lyx = group_sum<G>(Lyx);
  Lyy = group_sum<G>(Lyy);
  if (valid && g == 0) {
    float* o = L_out + 9 * I;
    o[0] = Lxx; o[1] = Lxy; o[2] = 0.f;
    o[3] = Lyx; o[4] = Lyy; o[5] = 0.f;
    o[6] = 0.f; o[7] = 0.f; o[8] = 0.f;
  }
}

// grid for one group of G lanes per item
inline int group_grid(int n_items, int threads, int G) {
  return static_cast<int>((static_cast<long long>(n_items) * G + threads - 1) / threads);
}

// the neighbour sums with their group sizes (densities always 16 lanes a
// particle; forces and gradients 16 in small systems, else 8)
void launch_density(const SphArgs& a, const double* stress, int T, cudaStream_t s) {
  if (a.n <= kTinySystem) sph_density<32><<<group_grid(a.n, T, 32), T, 0, s>>>(a, stress);
  else sph_density<16><<<group_grid(a.n, T, 16), T, 0, s>>>(a, stress);
}

void launch_force(const SphArgs& a, const double* stress, int T, cudaStream_t s) {
  if (a.n <= kTinySystem) sph_force<32><<<group_grid(a.n, T, 32), T, 0, s>>>(a, stress);
  else if (a.n <= kSmallSystem) sph_force<16><<<group_grid(a.n, T, 16), T, 0, s>>>(a, stress);
  else sph_force<8><<<group_grid(a.n, T, 8), T, 0, s>>>(a, stress);
}

void launch_velgrad(const SphArgs& a, float* L_out, int T, cudaStream_t s) {
  if (a.n_fluid <= 0) return;
  if (a.n <= kTinySystem) sph_velgrad<32><<<group_grid(a.n_fluid, T, 32), T, 0, s>>>(a, L_out);
  else if (a.n <= kSmallSystem) sph_velgrad<16><<<group_grid(a.n_fluid, T, 16), T, 0, s>>>(a, L_out);
  else sph_velgrad<8><<<group_grid(a.n_fluid, T, 8), T, 0, s>>>(a, L_out);
}

// systems whose cell list one block builds (scan, scatter, in-cell sort)
constexpr int kOneBlockParticles = 8192;
constexpr int kOneBlockCells = 8192;

// the cell list from the binned counts (cnt is zero again on exit)
void finish_cells(const SphArgs& a, cudaStream_t s) {
  const int T = 128;
  if (a.n <= kOneBlockParticles && a.ncell <= kOneBlockCells) {
    sph_cells_block<<<1, 1024, 0, s>>>(a);
    return;
  }
  sph_scan<<<1, 1024, 0, s>>>(a);
  sph_scatter<<<(a.n + T - 1) / T, T, 0, s>>>(a);
  sph_cellsort<<<static_cast<int>((32LL * a.ncell + T - 1) / T), T, 0, s>>>(a);
}

// cell list of the current positions (cnt is zero on entry and on exit)
void build_cells(const SphArgs& a, cudaStream_t s) {
  const int T = 128;
  sph_bin<<<(a.n + T - 1) / T, T, 0, s>>>(a);
  finish_cells(a, s);
}

}  // namespace

struct lhmm_sph_s {
  lhmm_sph_params p;
  SphArgs a;
  int threads = 128;
  cudaStream_t stream = nullptr;
};

namespace {

void free_sph(lhmm_sph_t h) {
  if (!h) return;
  cudaFree(h->a.pos);
  cudaFree(h->a.vel);
  cudaFree(h->a.acc);
  cudaFree(h->a.d);
  cudaFree(h->a.p);
  cudaFree(const_cast<int*>(h->a.wall));
  cudaFree(h->a.cnt);
  cudaFree(h->a.start);
  cudaFree(h->a.perm);
  cudaFree(h->a.cell_of);
  cudaFree(h->a.pterm);
  cudaFree(h->a.sterm);
  delete h;
}

bool one_block_cells(const SphArgs& a) {
  return a.n <= kOneBlockParticles && a.ncell <= kOneBlockCells;
}

size_t one_block_smem(const SphArgs& a) {
  return sizeof(int) * (2 * static_cast<size_t>(a.ncell) + 1 + static_cast<size_t>(a.n));
}

// the start of a substep: n_kicks half kicks, the drift if asked, and the
// cell list of the new positions (one block for small systems)
void substep_start(const SphArgs& a, float half_dt, int n_kicks, int drift, int T,
                   cudaStream_t s) {
  if (one_block_cells(a)) {
    sph_substep_cells_block<<<1, 1024, one_block_smem(a), s>>>(a, half_dt, n_kicks, drift);
    return;
  }
  sph_kick_drift_bin<<<(a.n + T - 1) / T, T, 0, s>>>(a, half_dt, n_kicks, drift);
  finish_cells(a, s);
}

// density and forces on the current cell list
cudaError_t forces_on_cells(lhmm_sph_s* h, const double* stress, cudaStream_t s) {
  launch_density(h->a, stress, h->threads, s);
  launch_force(h->a, stress, h->threads, s);
  return cudaGetLastError();
}

cudaError_t eval_forces(lhmm_sph_s* h, const double* stress, cudaStream_t s) {
  substep_start(h->a, 0.f, 0, 0, h->threads, s);
  return forces_on_cells(h, stress, s);
}

}  // namespace

extern "C" lhmm_status lhmm_sph_create(const lhmm_sph_params* params, const float* pos0_host,
                                       const float* vel0_host, void* stream, lhmm_sph_t* out) {
  if (!params || !out || !pos0_host || !vel0_host) return LHMM_ERR_ARG;
  *out = nullptr;
  const lhmm_sph_params& p = *params;
  if (p.n <= 0 || p.n_wall < 0 || p.n_wall > p.n || !(p.h > 0.f) || !(p.Lx >= 2.f * p.h) ||
      !(p.Ly >= 2.f * p.h) || !(p.mass > 0.f) || !(p.rho0 > 0.f) || !(p.dt > 0.f) ||
      (p.kernel != LHMM_SPH_WENDLAND_C2 && p.kernel != LHMM_SPH_LUCY))
    return LHMM_ERR_ARG;
  lhmm_sph_s* h = new lhmm_sph_s();
  h->p = p;
  h->stream = static_cast<cudaStream_t>(stream);
  SphArgs& a = h->a;
  a.n = p.n;
  a.n_fluid = p.n - p.n_wall;
  a.ncx = std::max(3, static_cast<int>(std::floor(p.Lx / p.h)));
  a.ncy = std::max(3, static_cast<int>(std::floor(p.Ly / p.h)));
  a.ncell = a.ncx * a.ncy;
  a.Lx = p.Lx;
  a.Ly = p.Ly;
  a.cwx = p.Lx / a.ncx;
  a.cwy = p.Ly / a.ncy;
  a.h = p.h;
  a.hinv = 1.f / p.h;
  a.mass = p.mass;
  a.rho0 = p.rho0;
  a.c2rho0_7 = p.c * p.c * p.rho0 / 7.f;
  a.pb = p.theta_pb * p.c * p.c * p.rho0 / 7.f;
  a.a_visc = 2.f * p.eta_s - p.zeta_s;
  a.b_visc = (p.visc_coeffs == LHMM_SPH_VISC_PAPER_LITERAL) ? 4.f * p.zeta_s + 2.f * p.eta_s
                                                            : 4.f * p.zeta_s;
  a.dt = p.dt;
  a.kernel = p.kernel;
  a.body_mode = p.body_mode;
  a.bfx = p.body_force[0];
  a.bfy = p.body_force[1];
  const size_t n = static_cast<size_t>(p.n);
  std::vector<int> wall(n, 0);
  for (size_t I = static_cast<size_t>(a.n_fluid); I < n; ++I) wall[I] = 1;  // walls come last
  cudaError_t e;
  int* wall_d = nullptr;
  if ((e = cudaMalloc(&a.pos, sizeof(float2) * n)) != cudaSuccess ||
      (e = cudaMalloc(&a.vel, sizeof(float2) * n)) != cudaSuccess ||
      (e = cudaMalloc(&a.acc, sizeof(float2) * n)) != cudaSuccess ||
      (e = cudaMalloc(&a.d, sizeof(float) * n)) != cudaSuccess ||
      (e = cudaMalloc(&a.p, sizeof(float) * n)) != cudaSuccess ||
      (e = cudaMalloc(&wall_d, sizeof(int) * n)) != cudaSuccess ||
      (e = cudaMalloc(&a.cnt, sizeof(int) * a.ncell)) != cudaSuccess ||
      (e = cudaMalloc(&a.start, sizeof(int) * (a.ncell + 1))) != cudaSuccess ||
      (e = cudaMalloc(&a.perm, sizeof(int) * n)) != cudaSuccess ||
      (e = cudaMalloc(&a.cell_of, sizeof(int) * n)) != cudaSuccess ||
      (e = cudaMalloc(&a.pterm, sizeof(float) * n)) != cudaSuccess ||
      (e = cudaMalloc(&a.sterm, sizeof(float4) * n)) != cudaSuccess) {
    a.wall = wall_d;
    free_sph(h);
    return lhmm_cuda_error(e);
  }
  a.wall = wall_d;
  std::vector<float2> pos(n), vel(n);
  for (size_t I = 0; I < n; ++I) {
    float x = pos0_host[2 * I], y = pos0_host[2 * I + 1];
    x -= p.Lx * std::floor(x / p.Lx);
    y -= p.Ly * std::floor(y / p.Ly);
    pos[I] = make_float2(x, y);
    vel[I] = wall[I] ? make_float2(0.f, 0.f) : make_float2(vel0_host[2 * I], vel0_host[2 * I + 1]);
  }
  cudaStream_t s = h->stream;
  if (one_block_cells(a) && one_block_smem(a) > 48 * 1024 &&
      (e = cudaFuncSetAttribute(sph_substep_cells_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(one_block_smem(a)))) != cudaSuccess) {
    free_sph(h);
    return lhmm_cuda_error(e);
  }
  if ((e = cudaMemcpyAsync(a.pos, pos.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(a.vel, vel.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(wall_d, wall.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(a.cnt, 0, sizeof(int) * a.ncell, s)) != cudaSuccess ||
      (e = eval_forces(h, nullptr, s)) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    free_sph(h);
    return lhmm_cuda_error(e);
  }
  *out = h;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_sph_destroy(lhmm_sph_t h) {
  if (!h) return LHMM_ERR_ARG;
  cudaDeviceSynchronize();
  free_sph(h);
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_sph_step(lhmm_sph_t h, const double* stress_dev, int n_substeps,
                                     float* L_out_dev, void* stream) {
  if (!h || n_substeps < 0) return LHMM_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int T = h->threads, G = (h->a.n + T - 1) / T;
  const float half = 0.5f * h->p.dt;
  // substep k: half kick, drift, bin (with substep k-1's closing half kick
  // folded in), cell list, density, forces; the last closing half kick
  // after the loop
  for (int k = 0; k < n_substeps; ++k) {
    substep_start(h->a, half, k > 0 ? 2 : 1, 1, T, s);
    LHMM_CK(forces_on_cells(h, stress_dev, s));
  }
  if (n_substeps > 0) sph_kick_drift<<<G, T, 0, s>>>(h->a, half, 0);
  if (L_out_dev) {
    if (n_substeps == 0) {  // density of the current positions
      build_cells(h->a, s);
      launch_density(h->a, nullptr, T, s);
    }
    launch_velgrad(h->a, L_out_dev, T, s);
  }
  LHMM_CK(cudaGetLastError());
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_sph_recompute_forces(lhmm_sph_t h, const double* stress_dev,
                                                 void* stream) {
  if (!h) return LHMM_ERR_ARG;
  LHMM_CK(eval_forces(h, stress_dev, static_cast<cudaStream_t>(stream)));
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_sph_info(lhmm_sph_t h, int* n, int* n_wall) {
  if (!h) return LHMM_ERR_ARG;
  if (n) *n = h->a.n;
  if (n_wall) *n_wall = h->a.n - h->a.n_fluid;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_sph_get_state(lhmm_sph_t h, float* pos_host, float* vel_host,
                                          float* acc_host, float* density_host) {
  if (!h) return LHMM_ERR_ARG;
  LHMM_CK(cudaDeviceSynchronize());
  const size_t n = static_cast<size_t>(h->a.n);
  if (pos_host) LHMM_CK(cudaMemcpy(pos_host, h->a.pos, sizeof(float2) * n, cudaMemcpyDeviceToHost));
  if (vel_host) LHMM_CK(cudaMemcpy(vel_host, h->a.vel, sizeof(float2) * n, cudaMemcpyDeviceToHost));
  if (acc_host) LHMM_CK(cudaMemcpy(acc_host, h->a.acc, sizeof(float2) * n, cudaMemcpyDeviceToHost));
  if (density_host) LHMM_CK(cudaMemcpy(density_host, h->a.d, sizeof(float) * n, cudaMemcpyDeviceToHost));
  return LHMM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free velocity-gradient export.
//
// Some callers cannot call cudaMalloc at the point where they need this
// result: code running inside another framework's memory pool or
// allocator-free section, real-time loops that must not touch the CUDA
// allocator, or plug-ins that may only use memory they are handed.  For them
// this entry point computes the same SPH number densities and velocity
// gradients as lhmm_sph_step(..., n_substeps = 0, L_out) but keeps all of its
// scratch (cell list, densities, pressures) in one fixed-size array in device
// global memory that belongs to this library.  The array is a file-scope
// __device__ variable, so every GPU that loads the library holds it until the
// process exits.  The caller passes inputs and outputs as usual.
namespace {

constexpr int kNoallocMaxParticles = LHMM_NOALLOC_MAX_PARTICLES;
constexpr int kNoallocMaxCells = LHMM_NOALLOC_MAX_CELLS;
// cell_of, perm, density, pressure (per particle) and counters, starts (per cell)
constexpr size_t kNoallocBytes =
    4 * sizeof(int) * static_cast<size_t>(kNoallocMaxParticles) +
    sizeof(int) * (2 * static_cast<size_t>(kNoallocMaxCells) + 64);

static __device__ __align__(256) unsigned char g_sph_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device.  The symbol's
// name is only a host-side handle; the address has to be looked up once per
// device (with that device current) before a kernel may use it.
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sph_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" lhmm_status lhmm_sph_velgrad_noalloc(const lhmm_sph_params* params,
                                                const float* pos_dev, const float* vel_dev,
                                                float* L_out_dev, void* stream) {
  if (!params || !pos_dev || !vel_dev || !L_out_dev) return LHMM_ERR_ARG;
  const lhmm_sph_params& p = *params;
  if (p.n <= 0 || p.n_wall < 0 || p.n_wall > p.n || !(p.h > 0.f) || !(p.Lx >= 2.f * p.h) ||
      !(p.Ly >= 2.f * p.h) || !(p.mass > 0.f) || !(p.rho0 > 0.f) ||
      (p.kernel != LHMM_SPH_WENDLAND_C2 && p.kernel != LHMM_SPH_LUCY))
    return LHMM_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(pos_dev) | reinterpret_cast<uintptr_t>(vel_dev)) % 8 != 0)
    return LHMM_ERR_ARG;  // read as float2
  const int ncx = std::max(3, static_cast<int>(std::floor(p.Lx / p.h)));
  const int ncy = std::max(3, static_cast<int>(std::floor(p.Ly / p.h)));
  if (p.n > kNoallocMaxParticles || static_cast<long long>(ncx) * ncy > kNoallocMaxCells)
    return LHMM_ERR_ARG;  // beyond the fixed scratch array
  void* base = nullptr;
  LHMM_CK(noalloc_scratch(&base));
  SphArgs a{};
  a.n = p.n;
  a.n_fluid = p.n - p.n_wall;
  a.ncx = ncx;
  a.ncy = ncy;
  a.ncell = ncx * ncy;
  a.Lx = p.Lx;
  a.Ly = p.Ly;
  a.cwx = p.Lx / ncx;
  a.cwy = p.Ly / ncy;
  a.h = p.h;
  a.hinv = 1.f / p.h;
  a.mass = p.mass;
  a.rho0 = p.rho0;
  a.c2rho0_7 = p.c * p.c * p.rho0 / 7.f;
  a.pb = p.theta_pb * p.c * p.c * p.rho0 / 7.f;
  a.kernel = p.kernel;
  a.pos = const_cast<float2*>(reinterpret_cast<const float2*>(pos_dev));
  a.vel = const_cast<float2*>(reinterpret_cast<const float2*>(vel_dev));
  int* ib = static_cast<int*>(base);
  a.cell_of = ib;
  a.perm = ib + kNoallocMaxParticles;
  a.d = reinterpret_cast<float*>(ib + 2 * kNoallocMaxParticles);
  a.p = reinterpret_cast<float*>(ib + 3 * kNoallocMaxParticles);
  a.cnt = ib + 4 * kNoallocMaxParticles;  // zeroed at the start of every call
  a.start = a.cnt + kNoallocMaxCells;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int T = 128;
  LHMM_CK(cudaMemsetAsync(a.cnt, 0, sizeof(int) * a.ncell, s));
  build_cells(a, s);
  launch_density(a, nullptr, T, s);
  launch_velgrad(a, L_out_dev, T, s);
  LHMM_CK(cudaGetLastError());
  return LHMM_OK;
}
