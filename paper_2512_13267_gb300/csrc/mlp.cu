// mlp.cu -- the learned stress closure of this library (not in the paper):
// an ensemble of MLPs (in -> hidden^L -> out, exact GELU) that predicts the
// polymer-stress increment of a micro-domain over one macro step from its
// velocity-gradient history and current stress.  BF16 operands on the tensor
// cores (mma.sync m16n8k16, FP32 accumulation), FP32 master weights, AdamW
// (Loshchilov & Hutter), all members of the ensemble in one launch (grid.z).
//
// Every product is one "NT" GEMM C[M x N] = A[M x K] . B[N x K]^T with both
// operands stored K-contiguous (row-major, leading dimension >= K):
//   forward    Z_l = H_{l-1} W_l^T           A = H_{l-1} [B x in],  B = W_l  [out x in]
//   dX         dH_{l-1} = dZ_l W_l            A = dZ_l    [B x out], B = W_l^T [in x out]
//   dW         dW_l = dZ_l^T H_{l-1}          A = dZ_l^T  [out x B], B = H^T   [in x B]
// so the forward epilogue also writes H^T and the backward epilogue dZ^T.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda.h>  // CUtensorMap and its enums (the encoder comes from the driver at run time)
#include <cuda_bf16.h>

#include "lhmm_common.cuh"

namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 128, BN = 128, BK = 32, SROW = BK + 8;  // padded smem rows: no ldmatrix conflicts
constexpr int GEMM_THREADS = 256;

enum { EPI_FWD_HIDDEN = 0, EPI_FWD_OUT = 1, EPI_BWD_DH = 2, EPI_DW = 3, EPI_FWD_INFER = 4 };

struct GemmArgs {
  const bf16* A;
  const bf16* B;
  int M, N, K, lda, ldb;
  long long sA, sB;  // per-member strides (elements)
  const float* bias;
  long long sBias;
  float* Cf;
  int ldc;
  long long sC;
  bf16* Hb;
  int ldh;
  long long sH;
  bf16* HTb;
  int ldht;
  long long sHT;
  const float* Zprev;
  int ldz;
  long long sZ;
  int k_split;
};

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// The fused epilogue of one element (m, n) of member `member` (the same for
// both GEMM kernels below).
template <int EPI>
__device__ __forceinline__ void store_epi(const GemmArgs& g, int member, int m, int n, float v) {
  if (EPI == EPI_DW) {
    float* c = g.Cf + g.sC * member + static_cast<long long>(m) * g.ldc + n;
    if (g.k_split > 1) atomicAdd(c, v);
    else *c = v;
  } else if (EPI == EPI_FWD_OUT) {
    v += g.bias[g.sBias * member + n];
    g.Cf[g.sC * member + static_cast<long long>(m) * g.ldc + n] = v;
  } else if (EPI == EPI_FWD_HIDDEN || EPI == EPI_FWD_INFER) {
    const float z = v + g.bias[g.sBias * member + n];
    const bf16 h = __float2bfloat16(gelu(z));
    g.Hb[g.sH * member + static_cast<long long>(m) * g.ldh + n] = h;
    if (EPI == EPI_FWD_HIDDEN) {
      g.Cf[g.sC * member + static_cast<long long>(m) * g.ldc + n] = z;
      g.HTb[g.sHT * member + static_cast<long long>(n) * g.ldht + m] = h;
    }
  } else {  // EPI_BWD_DH: dZ_{l-1} = dH_{l-1} * GELU'(Z_{l-1})
    const float z = g.Zprev[g.sZ * member + static_cast<long long>(m) * g.ldz + n];
    const bf16 dz = __float2bfloat16(v * gelu_grad(z));
    g.Hb[g.sH * member + static_cast<long long>(m) * g.ldh + n] = dz;
    g.HTb[g.sHT * member + static_cast<long long>(n) * g.ldht + m] = dz;
  }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldmatrix_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3,
                                            const void* smem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C = A . B^T on a 128 x 128 tile per block, 8 warps of 32 x 64, BK = 32,
// cp.async double buffer, ldmatrix fragment loads, fused epilogue.
template <int EPI>
__global__ void __launch_bounds__(GEMM_THREADS) gemm_nt(const GemmArgs g) {
  __shared__ __align__(16) bf16 sA[2][BM][SROW];
  __shared__ __align__(16) bf16 sB[2][BN][SROW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int member = blockIdx.z / g.k_split, split = blockIdx.z % g.k_split;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const bf16* A = g.A + g.sA * member;
  const bf16* B = g.B + g.sB * member;
  const int kc = ((g.K / BK + g.k_split - 1) / g.k_split) * BK;  // K per split
  const int kbeg = split * kc, kend = min(g.K, kbeg + kc);
  const int ktiles = kend > kbeg ? (kend - kbeg) / BK : 0;

  auto load_tile = [&](int stage, int k0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int c = tid + r * GEMM_THREADS;  // 512 16-byte chunks per operand tile
      const int row = c >> 2, ch = c & 3;
      const int gm = m0 + row, gn = n0 + row;
      const bf16* pa = A + static_cast<long long>(gm < g.M ? gm : 0) * g.lda + k0 + ch * 8;
      const bf16* pb = B + static_cast<long long>(gn < g.N ? gn : 0) * g.ldb + k0 + ch * 8;
      cp_async16(&sA[stage][row][ch * 8], pa, gm < g.M ? 16 : 0);
      cp_async16(&sB[stage][row][ch * 8], pb, gn < g.N ? 16 : 0);
    }
    cp_async_commit();
  };

  float acc[2][8][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

  if (ktiles > 0) load_tile(0, kbeg);
  for (int kt = 0; kt < ktiles; ++kt) {
    const int st = kt & 1;
    if (kt + 1 < ktiles) {
      load_tile(st ^ 1, kbeg + (kt + 1) * BK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned a[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i)
        ldmatrix_x4(a[i][0], a[i][1], a[i][2], a[i][3],
                    &sA[st][wm * 32 + i * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        unsigned b0, b1, b2, b3;
        ldmatrix_x4(b0, b1, b2, b3,
                    &sB[st][wn * 64 + p * 16 + (lane >> 4) * 8 + (lane & 7)][kk + ((lane >> 3) & 1) * 8]);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma_bf16(acc[i][2 * p], a[i], b0, b1);
          mma_bf16(acc[i][2 * p + 1], a[i], b2, b3);
        }
      }
    }
    __syncthreads();
  }

  // epilogue: fragment (i, j, q) holds row wm*32 + i*16 + lane/4 (+8 for q >= 2),
  // column wn*64 + j*8 + (lane%4)*2 + (q & 1)
#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm * 32 + i * 16 + (lane >> 2) + ((q >> 1) << 3);
        const int n = n0 + wn * 64 + j * 8 + ((lane & 3) << 1) + (q & 1);
        if (m >= g.M || n >= g.N) continue;
        store_epi<EPI>(g, member, m, n, acc[i][j][q]);
      }
    }
  }
}

template <int EPI>
cudaError_t run_gemm(const GemmArgs& g, int members, cudaStream_t s) {
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, members * g.k_split);
  gemm_nt<EPI><<<grid, GEMM_THREADS, 0, s>>>(g);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- tcgen05 path
// The same NT products on the fifth-generation tensor cores: per block a
// 128 x 128 tile of C, its FP32 accumulator in tensor memory (128 lanes x 128
// columns).  One thread issues everything asynchronous: TMA loads of 128-row
// x 64-column BF16 boxes of A and B (128-byte swizzle, zero fill past the
// matrix edges, one 3D tensor map per operand whose third axis is the
// ensemble member) into a ring of four stages, and per stage four
// tcgen05.mma (M = 128, N = 128, K = 16) whose completion frees the stage
// through tcgen05.commit.  Then the four warps copy their 32 accumulator
// rows (tcgen05.ld) into the stage memory, now idle, and the block runs the
// fused epilogue of gemm_nt from there: row-major outputs with the lanes of
// a warp along a row, transposed outputs (H^T, dZ^T) with the lanes along a
// column, so every store of a warp is contiguous.  Every wait on an mbarrier
// gives up after a bounded number of polls and raises a flag.
constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 3, TC_THREADS = 256;
constexpr int TC_LDT = TC_BN + 1;  // staged tile row stride (floats): conflict-free both ways
constexpr uint32_t TC_TILE_BYTES = TC_BM * TC_BK * 2;          // 16 KB per operand and stage
constexpr uint32_t TC_STAGE_BYTES = 2 * TC_TILE_BYTES;
constexpr size_t TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024;   // + room to align to 1024 B
constexpr uint32_t TC_WAIT_POLLS = 1u << 22;                    // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// wait for the phase of the given parity to complete; false after the poll limit
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < TC_WAIT_POLLS; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// shared-memory matrix descriptor of a K-major operand tile stored as the
// TMA's 128-byte swizzle writes it: rows of 128 bytes (64 BF16 along K),
// groups of 8 rows 1024 bytes apart; the start address steps 32 bytes per
// K = 16 inside a row
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);  // start address
  d |= static_cast<uint64_t>(1) << 16;                            // leading byte offset (16 B)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;                    // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                            // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                            // 128-byte swizzle
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 128, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                              (static_cast<uint32_t>(TC_BN >> 3) << 17) |
                              (static_cast<uint32_t>(TC_BM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kTcIdesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

static_assert(TC_BM * TC_LDT * 4 <= TC_STAGES * TC_STAGE_BYTES, "staged tile fits the stages");

// row pass of the fused epilogue for element (m, n), given its input `in`
// (the bias of column n, or Z_{l-1}(m, n) for the backward product): writes
// the row-major outputs and returns the value a transposed output takes (H
// or dZ, rounded to BF16) for the column pass
template <int EPI>
__device__ __forceinline__ float epi_row(const GemmArgs& g, int member, int m, int n, float v,
                                         float in) {
  if (EPI == EPI_DW) {
    float* c = g.Cf + g.sC * member + static_cast<long long>(m) * g.ldc + n;
    if (g.k_split > 1) atomicAdd(c, v);
    else *c = v;
    return 0.f;
  } else if (EPI == EPI_FWD_OUT) {
    g.Cf[g.sC * member + static_cast<long long>(m) * g.ldc + n] = v + in;
    return 0.f;
  } else if (EPI == EPI_FWD_HIDDEN || EPI == EPI_FWD_INFER) {
    const float z = v + in;
    const bf16 h = __float2bfloat16(gelu(z));
    g.Hb[g.sH * member + static_cast<long long>(m) * g.ldh + n] = h;
    if (EPI == EPI_FWD_HIDDEN) g.Cf[g.sC * member + static_cast<long long>(m) * g.ldc + n] = z;
    return __bfloat162float(h);
  } else {  // EPI_BWD_DH
    const bf16 dz = __float2bfloat16(v * gelu_grad(in));
    g.Hb[g.sH * member + static_cast<long long>(m) * g.ldh + n] = dz;
    return __bfloat162float(dz);
  }
}

template <int EPI>
__global__ void __launch_bounds__(TC_THREADS, 2)
    gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
            const GemmArgs g, int* err) {
  extern __shared__ unsigned char tc_smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * TC_STAGES + 1];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int member = blockIdx.z / g.k_split, split = blockIdx.z % g.k_split;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
  const int kt_all = (g.K + TC_BK - 1) / TC_BK;
  const int kt_per = (kt_all + g.k_split - 1) / g.k_split;
  const int kt0 = split * kt_per, nk = max(0, min(kt_all, kt0 + kt_per) - kt0);
  const uint32_t base = (smem_u32(tc_smem_raw) + 1023u) & ~1023u;  // swizzle atoms are 1024 B
  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[TC_STAGES]);
  const uint32_t done = smem_u32(&bars[2 * TC_STAGES]);
  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // 128 TMEM columns: the 128 x 128 FP32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TC_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  __shared__ int ok_s;
  if (tid == 0) {
    bool ok = true;
    int issued = 0;     // k-tiles whose loads were issued
    bool mma = false;   // whether any MMA was issued
    for (int it = 0; it < nk + TC_STAGES - 1 && ok; ++it) {
      if (it < nk) {  // produce k-tile `it`
        const int s = it % TC_STAGES;
        if (it >= TC_STAGES) ok = mbar_wait(empty0 + 8 * s, ((it / TC_STAGES) - 1) & 1);
        if (!ok) break;
        mbar_expect_tx(full0 + 8 * s, TC_STAGE_BYTES);
        const uint32_t sa = base + s * TC_STAGE_BYTES, sb = sa + TC_TILE_BYTES;
        const int kx = (kt0 + it) * TC_BK;
        tma_load_3d(sa, &mapA, full0 + 8 * s, kx, m0, member);
        tma_load_3d(sb, &mapB, full0 + 8 * s, kx, n0, member);
        issued = it + 1;
      }
      const int kc = it - (TC_STAGES - 1);
      if (kc >= 0) {  // consume k-tile kc
        const int s = kc % TC_STAGES;
        ok = mbar_wait(full0 + 8 * s, (kc / TC_STAGES) & 1);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = base + s * TC_STAGE_BYTES, sb = sa + TC_TILE_BYTES;
        const uint64_t da = umma_desc_sw128(sa), db = umma_desc_sw128(sb);
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk)  // +32 bytes per K = 16: +2 in the address field
          umma_bf16(tmem, da + 2 * kk, db + 2 * kk, (kc > 0 || kk > 0) ? 1u : 0u);
        umma_commit(empty0 + 8 * s);
        mma = true;
      }
    }
    // `done` completes when every MMA issued so far has (the epilogue waits
    // for it; on the error path it keeps TMEM alive until they finish)
    if (mma) umma_commit(done);
    if (!ok) {
      atomicExch(err, 1);
      if (mma) mbar_wait(done, 0);
      // and the loads already issued land before the block's memory goes away
      for (int k = 0; k < issued; ++k) mbar_wait(full0 + 8 * (k % TC_STAGES), (k / TC_STAGES) & 1);
    }
    ok_s = (ok && mma) ? 1 : 0;
  }
  __syncthreads();
  const bool have = ok_s && mbar_wait(done, 0);
  if (ok_s && !have) atomicExch(err, 1);
  // the accumulator tile, staged in the idle stage memory (all loads have
  // landed and every MMA has read its operands once `done` completed)
  float* const tile = reinterpret_cast<float*>(tc_smem_raw + (base - smem_u32(tc_smem_raw)));
  if (have) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // warp w may read TMEM lanes 32 (w % 4) .. + 31 (accumulator rows); the
    // two warps of a lane quarter split the columns
    const int r = 32 * (warp & 3) + lane;
    const int cbeg = (warp >> 2) * (TC_BN / 2);
    const uint32_t trow = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16);
#pragma unroll 1
    for (int c = cbeg; c < cbeg + TC_BN / 2; c += 16) {
      float v[16];
      tmem_ld16(trow + static_cast<uint32_t>(c), v);
#pragma unroll
      for (int k = 0; k < 16; ++k) tile[r * TC_LDT + c + k] = v[k];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (have) {
    // row pass: lanes along n, four rows at a time with their inputs loaded
    // ahead of the arithmetic (the bias once per column)
    constexpr int NJ = TC_BN / 32, RB = 4;
    float bias[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int n = n0 + 32 * j + lane;
      bias[j] = (EPI != EPI_DW && EPI != EPI_BWD_DH && n < g.N) ? g.bias[g.sBias * member + n] : 0.f;
    }
    const float* __restrict__ zp = g.Zprev + (EPI == EPI_BWD_DH ? g.sZ * member : 0);
    for (int r0 = warp * RB; r0 < TC_BM; r0 += RB * (TC_THREADS / 32)) {
      float in[RB][NJ];
#pragma unroll
      for (int rr = 0; rr < RB; ++rr)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const int m = m0 + r0 + rr, n = n0 + 32 * j + lane;
          in[rr][j] = bias[j];
          if (EPI == EPI_BWD_DH)
            in[rr][j] = (m < g.M && n < g.N) ? zp[static_cast<long long>(m) * g.ldz + n] : 0.f;
        }
#pragma unroll
      for (int rr = 0; rr < RB; ++rr) {
        const int r = r0 + rr, m = m0 + r;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const int nl = 32 * j + lane, n = n0 + nl;
          if (n < g.N)
            tile[r * TC_LDT + nl] = epi_row<EPI>(g, member, m, n, tile[r * TC_LDT + nl], in[rr][j]);
        }
      }
    }
    if (EPI == EPI_FWD_HIDDEN || EPI == EPI_BWD_DH) {  // column pass: lanes along m
      __syncthreads();
      for (int nl = warp; nl < TC_BN; nl += TC_THREADS / 32) {
        const int n = n0 + nl;
        if (n >= g.N) continue;
#pragma unroll
        for (int j = 0; j < TC_BM / 32; ++j) {
          const int r = 32 * j + lane, m = m0 + r;
          if (m < g.M)
            g.HTb[g.sHT * member + static_cast<long long>(n) * g.ldht + m] =
                __float2bfloat16(tile[r * TC_LDT + nl]);
        }
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN)
                 : "memory");
  }
}

// cuTensorMapEncodeTiled from the driver (no link against libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3D map (K, rows, member) of a K-major BF16 operand with leading dimension
// ld and member stride sm (elements), boxes of 64 x 128 x 1
bool make_map(CUtensorMap* map, const bf16* ptr, int K, int rows, int ld, long long sm, int members) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || (ld * 2) % 16 || (sm * 2) % 16) return false;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows),
                              static_cast<cuuint64_t>(members)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld) * 2, static_cast<cuuint64_t>(sm) * 2};
  const cuuint32_t box[3] = {TC_BK, TC_BM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t tc_attributes() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(gemm_tc<EPI_FWD_HIDDEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(TC_SMEM))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(gemm_tc<EPI_FWD_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(TC_SMEM))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(gemm_tc<EPI_BWD_DH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(TC_SMEM))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(gemm_tc<EPI_DW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(TC_SMEM))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(gemm_tc<EPI_FWD_INFER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(TC_SMEM))) != cudaSuccess)
    return e;
  return cudaSuccess;
}

template <int EPI>
cudaError_t run_gemm_tc(const GemmArgs& g, int members, int* err, cudaStream_t s) {
  CUtensorMap ma, mb;
  if (!make_map(&ma, g.A, g.K, g.M, g.lda, g.sA, members) ||
      !make_map(&mb, g.B, g.K, g.N, g.ldb, g.sB, members))
    return cudaErrorInvalidValue;
  dim3 grid((g.N + TC_BN - 1) / TC_BN, (g.M + TC_BM - 1) / TC_BM, members * g.k_split);
  gemm_tc<EPI><<<grid, TC_THREADS, TC_SMEM, s>>>(ma, mb, g, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- small kernels
// rows of X (fp32, ld in_dim) -> normalised bf16 X [B x in_pad] and X^T [in_pad x B]
__global__ void prep_input(const float* X, const int* rows, int B, int in_dim, int in_pad,
                           const float* mean, const float* inv_std, bf16* Xb, bf16* XTb,
                           long long member_rows_stride) {
  const int member = blockIdx.y;
  const long long total = static_cast<long long>(B) * in_pad;
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(t / in_pad), k = static_cast<int>(t % in_pad);
    float v = 0.f;
    if (k < in_dim) {
      const long long r = rows ? rows[member * member_rows_stride + b] : b;
      v = (X[r * in_dim + k] - mean[k]) * inv_std[k];
    }
    const bf16 h = __float2bfloat16(v);
    Xb[(static_cast<long long>(member) * B + b) * in_pad + k] = h;
    XTb[(static_cast<long long>(member) * in_pad + k) * B + b] = h;
  }
}

// loss = mean over batch and outputs of (y - t)^2 (targets scaled by out_scale);
// dY = 2 (y - t) / (B out) as bf16 [B x out_pad] and dY^T [out_pad x B]
__global__ void loss_grad(const float* Y, int ldy, const float* T, const int* rows, int B,
                          int out_dim, int out_pad, const float* inv_out_scale, bf16* dY, bf16* dYT,
                          float* loss, long long member_rows_stride) {
  const int member = blockIdx.y;
  const long long total = static_cast<long long>(B) * out_pad;
  float local = 0.f;
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(t / out_pad), o = static_cast<int>(t % out_pad);
    float d = 0.f;
    if (o < out_dim) {
      const long long r = rows ? rows[member * member_rows_stride + b] : b;
      const float e = Y[(static_cast<long long>(member) * B + b) * ldy + o] - T[r * out_dim + o] * inv_out_scale[o];
      local += e * e;
      d = 2.f * e / static_cast<float>(B * out_dim);
    }
    const bf16 h = __float2bfloat16(d);
    dY[(static_cast<long long>(member) * B + b) * out_pad + o] = h;
    dYT[(static_cast<long long>(member) * out_pad + o) * B + b] = h;
  }
  local = lhmm::warp_sum(local);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(&loss[member], local / static_cast<float>(B * out_dim));
}

// db[member][n] = sum_b dZ^T[member][n][b]
__global__ void bias_grad(const bf16* dZT, int N, int B, long long sZT, float* db, long long sdb) {
  const int member = blockIdx.y;
  const int n = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (n >= N) return;
  const bf16* row = dZT + sZT * member + static_cast<long long>(n) * B;
  float s = 0.f;
  for (int b = threadIdx.x & 31; b < B; b += 32) s += __bfloat162float(row[b]);
  s = lhmm::warp_sum(s);
  if ((threadIdx.x & 31) == 0) db[sdb * member + n] = s;
}

// AdamW on the fp32 master parameters of all members, then bf16 copies
// W [out x in] and W^T [in x out] of every weight matrix
struct LayerMap {
  int n_layers;
  int out_pad[8], in_pad[8];
  long long w_off[8], b_off[8];    // offsets in the per-member parameter vector
  long long wb_off[8], wt_off[8];  // offsets in the per-member bf16 buffers
};

__global__ void adamw(float* P, const float* G, float* Mo, float* V, long long n_per, int members,
                      float lr, float b1, float b2, float eps, float wd, float bc1, float bc2,
                      const unsigned char* decay_mask) {
  const long long total = n_per * members;
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float g = G[t];
    const float m = b1 * Mo[t] + (1.f - b1) * g;
    const float v = b2 * V[t] + (1.f - b2) * g * g;
    Mo[t] = m;
    V[t] = v;
    const float w = decay_mask[t % n_per] ? wd : 0.f;
    P[t] = P[t] * (1.f - lr * w) - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
  }
}

__global__ void to_bf16_weights(const float* P, long long n_per, bf16* Wb, bf16* WTb,
                                long long nb_per, LayerMap L) {
  const int member = blockIdx.y;
  for (int l = 0; l < L.n_layers; ++l) {
    const int O = L.out_pad[l], I = L.in_pad[l];
    const float* W = P + member * n_per + L.w_off[l];
    bf16* wb = Wb + member * nb_per + L.wb_off[l];
    bf16* wt = WTb + member * nb_per + L.wt_off[l];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < O * I; t += gridDim.x * blockDim.x) {
      const int o = t / I, i = t % I;
      const bf16 h = __float2bfloat16(W[t]);
      wb[t] = h;
      wt[static_cast<long long>(i) * O + o] = h;
    }
  }
}

// mean and relative spread of the ensemble predictions (scaled back to stress units)
__global__ void ensemble_stats(const float* Y, int ldy, long long sY, int members, int n,
                               int out_dim, const float* out_scale, float* mean, float* spread) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  float mu[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int m = 0; m < members; ++m)
    for (int o = 0; o < out_dim; ++o) mu[o] += Y[sY * m + static_cast<long long>(I) * ldy + o] * out_scale[o];
  for (int o = 0; o < out_dim; ++o) mu[o] /= static_cast<float>(members);
  float var = 0.f;
  for (int m = 0; m < members; ++m)
    for (int o = 0; o < out_dim; ++o) {
      const float d = Y[sY * m + static_cast<long long>(I) * ldy + o] * out_scale[o] - mu[o];
      var += d * d;
    }
  var /= static_cast<float>(members > 1 ? members - 1 : 1);
  for (int o = 0; o < out_dim; ++o) mean[static_cast<long long>(I) * out_dim + o] = mu[o];
  spread[I] = sqrtf(var);
}

}  // namespace

// ---------------------------------------------------------------- handle
struct lhmm_closure_s {
  int members = 0, in_dim = 0, hidden = 0, n_hidden = 0, out_dim = 0, in_pad = 0;
  int out_pad = 32;  // output layer padded to one k-tile, so dX of that layer is a whole tile
  int n_layers = 0;
  LayerMap L{};
  long long n_per = 0, nb_per = 0;  // fp32 params and bf16 weight elements per member
  float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
  unsigned char* decay = nullptr;
  bf16 *Wb = nullptr, *WTb = nullptr;
  float *in_mean = nullptr, *in_istd = nullptr, *out_scale = nullptr, *out_iscale = nullptr;
  long long step = 0;
  // activation workspace, sized for `cap` rows
  int cap = 0;
  bf16 *Xb = nullptr, *XTb = nullptr, *dYb = nullptr, *dYTb = nullptr;
  std::vector<bf16*> Hb, HTb, dZb, dZTb;
  std::vector<float*> Z;
  float* Y = nullptr;
  float* loss = nullptr;
  int gemm_path = 1;     // 1: tcgen05 + TMA (gemm_tc), 0: mma.sync (gemm_nt)
  int* tc_err = nullptr; // set by gemm_tc when a bounded wait gives up
};

namespace {

void free_ws(lhmm_closure_s* c) {
  cudaFree(c->Xb);
  cudaFree(c->XTb);
  cudaFree(c->dYb);
  cudaFree(c->dYTb);
  cudaFree(c->Y);
  for (auto* p : c->Hb) cudaFree(p);
  for (auto* p : c->HTb) cudaFree(p);
  for (auto* p : c->dZb) cudaFree(p);
  for (auto* p : c->dZTb) cudaFree(p);
  for (auto* p : c->Z) cudaFree(p);
  c->Hb.clear();
  c->HTb.clear();
  c->dZb.clear();
  c->dZTb.clear();
  c->Z.clear();
  c->Xb = c->XTb = c->dYb = c->dYTb = nullptr;
  c->Y = nullptr;
  c->cap = 0;
}

void free_closure(lhmm_closure_s* c) {
  if (!c) return;
  free_ws(c);
  cudaFree(c->P);
  cudaFree(c->G);
  cudaFree(c->M);
  cudaFree(c->V);
  cudaFree(c->decay);
  cudaFree(c->Wb);
  cudaFree(c->WTb);
  cudaFree(c->in_mean);
  cudaFree(c->in_istd);
  cudaFree(c->out_scale);
  cudaFree(c->out_iscale);
  cudaFree(c->loss);
  cudaFree(c->tc_err);
  delete c;
}

cudaError_t ensure_ws(lhmm_closure_s* c, int rows) {
  if (rows <= c->cap) return cudaSuccess;
  free_ws(c);
  const size_t R = static_cast<size_t>(rows), Mm = static_cast<size_t>(c->members);
  const size_t H = static_cast<size_t>(c->hidden);
  cudaError_t e;
  if ((e = cudaMalloc(&c->Xb, sizeof(bf16) * Mm * R * c->in_pad)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->XTb, sizeof(bf16) * Mm * R * c->in_pad)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->dYb, sizeof(bf16) * Mm * R * c->out_pad)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->dYTb, sizeof(bf16) * Mm * R * c->out_pad)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->Y, sizeof(float) * Mm * R * c->out_pad)) != cudaSuccess) return e;
  for (int l = 0; l < c->n_hidden; ++l) {
    bf16 *h, *ht, *dz, *dzt;
    float* z;
    if ((e = cudaMalloc(&h, sizeof(bf16) * Mm * R * H)) != cudaSuccess) return e;
    c->Hb.push_back(h);
    if ((e = cudaMalloc(&ht, sizeof(bf16) * Mm * R * H)) != cudaSuccess) return e;
    c->HTb.push_back(ht);
    if ((e = cudaMalloc(&dz, sizeof(bf16) * Mm * R * H)) != cudaSuccess) return e;
    c->dZb.push_back(dz);
    if ((e = cudaMalloc(&dzt, sizeof(bf16) * Mm * R * H)) != cudaSuccess) return e;
    c->dZTb.push_back(dzt);
    if ((e = cudaMalloc(&z, sizeof(float) * Mm * R * H)) != cudaSuccess) return e;
    c->Z.push_back(z);
  }
  c->cap = rows;
  return cudaSuccess;
}

template <int EPI>
cudaError_t gemm(const lhmm_closure_s* c, const GemmArgs& g, cudaStream_t s) {
  return c->gemm_path == 1 ? run_gemm_tc<EPI>(g, c->members, c->tc_err, s)
                           : run_gemm<EPI>(g, c->members, s);
}

// forward over `rows` inputs already in Xb/XTb; train=1 keeps Z and H^T
cudaError_t forward(lhmm_closure_s* c, int rows, bool train, cudaStream_t s) {
  const long long R = rows, Hd = c->hidden;
  for (int l = 0; l < c->n_layers; ++l) {
    const bool last = (l == c->n_layers - 1);
    GemmArgs g{};
    g.A = (l == 0) ? c->Xb : c->Hb[l - 1];
    g.lda = (l == 0) ? c->in_pad : c->hidden;
    g.sA = R * g.lda;
    g.B = c->Wb + c->L.wb_off[l];
    g.ldb = c->L.in_pad[l];
    g.sB = c->nb_per;
    g.M = rows;
    g.N = c->L.out_pad[l];
    g.K = c->L.in_pad[l];
    g.bias = c->P + c->L.b_off[l];
    g.sBias = c->n_per;
    g.k_split = 1;
    cudaError_t e;
    if (last) {
      g.Cf = c->Y;
      g.ldc = c->out_pad;
      g.sC = R * c->out_pad;
      e = gemm<EPI_FWD_OUT>(c, g, s);
    } else {
      g.Hb = c->Hb[l];
      g.ldh = c->hidden;
      g.sH = R * Hd;
      g.HTb = c->HTb[l];
      g.ldht = rows;
      g.sHT = R * Hd;
      g.Cf = c->Z[l];
      g.ldc = c->hidden;
      g.sC = R * Hd;
      e = train ? gemm<EPI_FWD_HIDDEN>(c, g, s) : gemm<EPI_FWD_INFER>(c, g, s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// backward from dY (in dYb/dYTb) into G
cudaError_t backward(lhmm_closure_s* c, int rows, cudaStream_t s) {
  const long long R = rows, Hd = c->hidden;
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->G, 0, sizeof(float) * c->n_per * c->members, s)) != cudaSuccess) return e;
  for (int l = c->n_layers - 1; l >= 0; --l) {
    const bf16* dZ = (l == c->n_layers - 1) ? c->dYb : c->dZb[l];
    const bf16* dZT = (l == c->n_layers - 1) ? c->dYTb : c->dZTb[l];
    const int Np = c->L.out_pad[l];
    const long long sdz = R * Np;
    // dW_l = dZ_l^T H_{l-1}  (M = out, N = in, K = rows), split over K
    GemmArgs g{};
    g.A = dZT;
    g.lda = rows;
    g.sA = sdz;
    g.B = (l == 0) ? c->XTb : c->HTb[l - 1];
    g.ldb = rows;
    g.sB = (l == 0) ? R * c->in_pad : R * Hd;
    g.M = Np;
    g.N = c->L.in_pad[l];
    g.K = rows;
    g.Cf = c->G + c->L.w_off[l];
    g.ldc = c->L.in_pad[l];
    g.sC = c->n_per;
    g.k_split = std::max(1, std::min(16, rows / 512));
    if ((e = gemm<EPI_DW>(c, g, s)) != cudaSuccess) return e;
    // db_l = column sums of dZ_l
    {
      dim3 grid((Np + 7) / 8, c->members);
      bias_grad<<<grid, 256, 0, s>>>(dZT, Np, rows, sdz, c->G + c->L.b_off[l], c->n_per);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (l == 0) break;
    // dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1})  (M = rows, N = in = hidden, K = out)
    GemmArgs h{};
    h.A = dZ;
    h.lda = Np;
    h.sA = sdz;
    h.B = c->WTb + c->L.wt_off[l];
    h.ldb = Np;
    h.sB = c->nb_per;
    h.M = rows;
    h.N = c->hidden;
    h.K = Np;
    h.Zprev = c->Z[l - 1];
    h.ldz = c->hidden;
    h.sZ = R * Hd;
    h.Hb = c->dZb[l - 1];
    h.ldh = c->hidden;
    h.sH = R * Hd;
    h.HTb = c->dZTb[l - 1];
    h.ldht = rows;
    h.sHT = R * Hd;
    h.k_split = 1;
    if ((e = gemm<EPI_BWD_DH>(c, h, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t refresh_bf16(lhmm_closure_s* c, cudaStream_t s) {
  dim3 grid(64, c->members);
  to_bf16_weights<<<grid, 256, 0, s>>>(c->P, c->n_per, c->Wb, c->WTb, c->nb_per, c->L);
  return cudaGetLastError();
}

}  // namespace

extern "C" lhmm_status lhmm_closure_create(int members, int in_dim, int hidden, int n_hidden,
                                           int out_dim, uint64_t seed, lhmm_closure_t* out) {
  if (!out || members < 1 || members > 16 || in_dim < 1 || hidden < 32 || hidden % 32 != 0 ||
      n_hidden < 1 || n_hidden > 6 || out_dim < 1 || out_dim > 8)
    return LHMM_ERR_ARG;
  *out = nullptr;
  lhmm_closure_s* c = new lhmm_closure_s();
  c->members = members;
  c->in_dim = in_dim;
  c->hidden = hidden;
  c->n_hidden = n_hidden;
  c->out_dim = out_dim;
  c->in_pad = (in_dim + 31) / 32 * 32;
  c->n_layers = n_hidden + 1;
  LayerMap& L = c->L;
  L.n_layers = c->n_layers;
  long long off = 0, boff = 0;
  for (int l = 0; l < c->n_layers; ++l) {
    L.in_pad[l] = (l == 0) ? c->in_pad : hidden;
    L.out_pad[l] = (l == c->n_layers - 1) ? c->out_pad : hidden;
    L.w_off[l] = off;
    off += static_cast<long long>(L.out_pad[l]) * L.in_pad[l];
    L.b_off[l] = off;
    off += L.out_pad[l];
    L.wb_off[l] = boff;
    L.wt_off[l] = boff;  // W and W^T live in separate buffers with the same offsets
    boff += static_cast<long long>(L.out_pad[l]) * L.in_pad[l];
  }
  c->n_per = off;
  c->nb_per = boff;
  const size_t np = static_cast<size_t>(c->n_per) * members;
  cudaError_t e;
  if ((e = cudaMalloc(&c->P, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMalloc(&c->G, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMalloc(&c->M, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMalloc(&c->V, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMalloc(&c->decay, c->n_per)) != cudaSuccess ||
      (e = cudaMalloc(&c->Wb, sizeof(bf16) * c->nb_per * members)) != cudaSuccess ||
      (e = cudaMalloc(&c->WTb, sizeof(bf16) * c->nb_per * members)) != cudaSuccess ||
      (e = cudaMalloc(&c->in_mean, sizeof(float) * in_dim)) != cudaSuccess ||
      (e = cudaMalloc(&c->in_istd, sizeof(float) * in_dim)) != cudaSuccess ||
      (e = cudaMalloc(&c->out_scale, sizeof(float) * 8)) != cudaSuccess ||
      (e = cudaMalloc(&c->out_iscale, sizeof(float) * 8)) != cudaSuccess ||
      (e = cudaMalloc(&c->loss, sizeof(float) * 16)) != cudaSuccess ||
      (e = cudaMalloc(&c->tc_err, sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(c->tc_err, 0, sizeof(int))) != cudaSuccess ||
      (e = tc_attributes()) != cudaSuccess) {
    free_closure(c);
    return lhmm_cuda_error(e);
  }
  // He-style init from a seeded host generator (splitmix64 -> Box-Muller);
  // padding rows/columns and biases start at zero; weights decay, biases do not
  std::vector<float> P(np, 0.f);
  std::vector<unsigned char> decay(static_cast<size_t>(c->n_per), 0);
  uint64_t st = seed ? seed : 0x9E3779B97F4A7C15ull;
  auto next = [&st]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto normal = [&]() {
    const double u1 = (static_cast<double>(next() >> 11) + 0.5) * 0x1p-53;
    const double u2 = (static_cast<double>(next() >> 11) + 0.5) * 0x1p-53;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  for (int m = 0; m < members; ++m) {
    for (int l = 0; l < c->n_layers; ++l) {
      const int O = (l == c->n_layers - 1) ? out_dim : hidden;
      const int I = (l == 0) ? in_dim : hidden;
      const double sd = std::sqrt(2.0 / I) * ((l == c->n_layers - 1) ? 0.5 : 1.0);
      for (int o = 0; o < O; ++o)
        for (int i = 0; i < I; ++i)
          P[m * c->n_per + L.w_off[l] + static_cast<long long>(o) * L.in_pad[l] + i] =
              static_cast<float>(normal() * sd);
    }
  }
  for (int l = 0; l < c->n_layers; ++l)
    for (long long k = L.w_off[l]; k < L.b_off[l]; ++k) decay[k] = 1;
  std::vector<float> ones(8, 1.f), zeros(static_cast<size_t>(in_dim), 0.f),
      ones_in(static_cast<size_t>(in_dim), 1.f);
  if ((e = cudaMemcpy(c->P, P.data(), sizeof(float) * np, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(c->M, 0, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMemset(c->V, 0, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMemset(c->G, 0, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMemcpy(c->decay, decay.data(), c->n_per, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->in_mean, zeros.data(), sizeof(float) * in_dim, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->in_istd, ones_in.data(), sizeof(float) * in_dim, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->out_scale, ones.data(), sizeof(float) * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->out_iscale, ones.data(), sizeof(float) * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = refresh_bf16(c, nullptr)) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) {
    free_closure(c);
    return lhmm_cuda_error(e);
  }
  *out = c;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_closure_destroy(lhmm_closure_t c) {
  if (!c) return LHMM_ERR_ARG;
  cudaDeviceSynchronize();
  free_closure(c);
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_closure_set_normalization(lhmm_closure_t c, const float* in_mean_host,
                                                      const float* in_std_host,
                                                      const float* out_scale_host) {
  if (!c || !in_mean_host || !in_std_host || !out_scale_host) return LHMM_ERR_ARG;
  std::vector<float> istd(static_cast<size_t>(c->in_dim)), os(8, 1.f), ios(8, 1.f);
  for (int k = 0; k < c->in_dim; ++k) {
    if (!(in_std_host[k] > 0.f)) return LHMM_ERR_ARG;
    istd[k] = 1.f / in_std_host[k];
  }
  for (int o = 0; o < c->out_dim; ++o) {
    if (!(out_scale_host[o] > 0.f)) return LHMM_ERR_ARG;
    os[o] = out_scale_host[o];
    ios[o] = 1.f / out_scale_host[o];
  }
  LHMM_CK(cudaMemcpy(c->in_mean, in_mean_host, sizeof(float) * c->in_dim, cudaMemcpyHostToDevice));
  LHMM_CK(cudaMemcpy(c->in_istd, istd.data(), sizeof(float) * c->in_dim, cudaMemcpyHostToDevice));
  LHMM_CK(cudaMemcpy(c->out_scale, os.data(), sizeof(float) * 8, cudaMemcpyHostToDevice));
  LHMM_CK(cudaMemcpy(c->out_iscale, ios.data(), sizeof(float) * 8, cudaMemcpyHostToDevice));
  return LHMM_OK;
}

// one AdamW step of every member on its own batch: rows_dev (members x B
// row indices into X/T, or NULL = rows 0..B-1 for every member)
extern "C" lhmm_status lhmm_closure_train_step(lhmm_closure_t c, const float* X_dev,
                                               const float* T_dev, const int* rows_dev, int B,
                                               float lr, float weight_decay, float* loss_dev,
                                               void* stream) {
  if (!c || !X_dev || !T_dev || B < 32 || B % 32 != 0) return LHMM_ERR_ARG;  // K of the dW product
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LHMM_CK(ensure_ws(c, B));
  const int members = c->members;
  dim3 g1(std::min(1024, (B * c->in_pad + 255) / 256), members);
  prep_input<<<g1, 256, 0, s>>>(X_dev, rows_dev, B, c->in_dim, c->in_pad, c->in_mean, c->in_istd,
                                c->Xb, c->XTb, B);
  LHMM_CK(cudaGetLastError());
  LHMM_CK(forward(c, B, true, s));
  LHMM_CK(cudaMemsetAsync(c->loss, 0, sizeof(float) * members, s));
  dim3 g2(std::min(1024, (B * c->out_pad + 255) / 256), members);
  loss_grad<<<g2, 256, 0, s>>>(c->Y, c->out_pad, T_dev, rows_dev, B, c->out_dim, c->out_pad,
                               c->out_iscale, c->dYb, c->dYTb, c->loss, B);
  LHMM_CK(cudaGetLastError());
  LHMM_CK(backward(c, B, s));
  if (lr > 0.f) {
    ++c->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - static_cast<float>(std::pow(b1, static_cast<double>(c->step)));
    const float bc2 = 1.f - static_cast<float>(std::pow(b2, static_cast<double>(c->step)));
    adamw<<<1024, 256, 0, s>>>(c->P, c->G, c->M, c->V, c->n_per, members, lr, b1, b2, 1e-8f,
                               weight_decay, bc1, bc2, c->decay);
    LHMM_CK(cudaGetLastError());
    LHMM_CK(refresh_bf16(c, s));
  }
  if (loss_dev) LHMM_CK(cudaMemcpyAsync(loss_dev, c->loss, sizeof(float) * members, cudaMemcpyDeviceToDevice, s));
  return LHMM_OK;
}

// ensemble mean prediction (n x out_dim, stress units) and spread (n): the
// sample standard deviation over members of the full output vector
extern "C" lhmm_status lhmm_closure_infer(lhmm_closure_t c, const float* X_dev, int n,
                                          float* mean_dev, float* spread_dev, void* stream) {
  if (!c || !X_dev || !mean_dev || !spread_dev || n < 0) return LHMM_ERR_ARG;
  if (n == 0) return LHMM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LHMM_CK(ensure_ws(c, n));
  dim3 g1(std::min(1024, (n * c->in_pad + 255) / 256), c->members);
  prep_input<<<g1, 256, 0, s>>>(X_dev, nullptr, n, c->in_dim, c->in_pad, c->in_mean, c->in_istd,
                                c->Xb, c->XTb, 0);
  LHMM_CK(cudaGetLastError());
  LHMM_CK(forward(c, n, false, s));
  ensemble_stats<<<(n + 127) / 128, 128, 0, s>>>(c->Y, c->out_pad, static_cast<long long>(n) * c->out_pad,
                                                 c->members, n, c->out_dim, c->out_scale, mean_dev,
                                                 spread_dev);
  LHMM_CK(cudaGetLastError());
  return LHMM_OK;
}

// raw (normalised-unit) outputs of every member for n inputs: members x n x out_dim
extern "C" lhmm_status lhmm_closure_forward(lhmm_closure_t c, const float* X_dev, int n,
                                            float* Y_host) {
  if (!c || !X_dev || !Y_host || n < 1) return LHMM_ERR_ARG;
  LHMM_CK(ensure_ws(c, n));
  dim3 g1(std::min(1024, (n * c->in_pad + 255) / 256), c->members);
  prep_input<<<g1, 256>>>(X_dev, nullptr, n, c->in_dim, c->in_pad, c->in_mean, c->in_istd, c->Xb,
                          c->XTb, 0);
  LHMM_CK(cudaGetLastError());
  LHMM_CK(forward(c, n, false, nullptr));
  std::vector<float> Y(static_cast<size_t>(c->members) * n * c->out_pad);
  LHMM_CK(cudaDeviceSynchronize());
  LHMM_CK(cudaMemcpy(Y.data(), c->Y, sizeof(float) * Y.size(), cudaMemcpyDeviceToHost));
  for (int m = 0; m < c->members; ++m)
    for (int i = 0; i < n; ++i)
      for (int o = 0; o < c->out_dim; ++o)
        Y_host[(static_cast<size_t>(m) * n + i) * c->out_dim + o] =
            Y[(static_cast<size_t>(m) * n + i) * c->out_pad + o];
  return LHMM_OK;
}

// parameters of one member in the unpadded layout W_0, b_0, W_1, b_1, ...
// (W_l row-major out x in); get copies the fp32 master, gradient the last
// gradient computed by lhmm_closure_train_step
static lhmm_status copy_member(lhmm_closure_t c, int member, float* host, bool to_device,
                               const float* src_dev) {
  if (!c || !host || member < 0 || member >= c->members) return LHMM_ERR_ARG;
  std::vector<float> buf(static_cast<size_t>(c->n_per));
  const float* base = src_dev ? src_dev : c->P;
  LHMM_CK(cudaDeviceSynchronize());
  LHMM_CK(cudaMemcpy(buf.data(), base + member * c->n_per, sizeof(float) * c->n_per, cudaMemcpyDeviceToHost));
  long long k = 0;
  for (int l = 0; l < c->n_layers; ++l) {
    const int O = (l == c->n_layers - 1) ? c->out_dim : c->hidden;
    const int I = (l == 0) ? c->in_dim : c->hidden;
    for (int o = 0; o < O; ++o)
      for (int i = 0; i < I; ++i) {
        float& d = buf[c->L.w_off[l] + static_cast<long long>(o) * c->L.in_pad[l] + i];
        if (to_device) d = host[k++];
        else host[k++] = d;
      }
    for (int o = 0; o < O; ++o) {
      float& d = buf[c->L.b_off[l] + o];
      if (to_device) d = host[k++];
      else host[k++] = d;
    }
  }
  if (to_device) {
    LHMM_CK(cudaMemcpy(c->P + member * c->n_per, buf.data(), sizeof(float) * c->n_per, cudaMemcpyHostToDevice));
    cudaError_t e = refresh_bf16(c, nullptr);
    if (e != cudaSuccess) return lhmm_cuda_error(e);
    LHMM_CK(cudaDeviceSynchronize());
  }
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_closure_get_params(lhmm_closure_t c, int member, float* host) {
  return copy_member(c, member, host, false, nullptr);
}
extern "C" lhmm_status lhmm_closure_set_params(lhmm_closure_t c, int member, const float* host) {
  return copy_member(c, member, const_cast<float*>(host), true, nullptr);
}
extern "C" lhmm_status lhmm_closure_get_grad(lhmm_closure_t c, int member, float* host) {
  if (!c) return LHMM_ERR_ARG;
  return copy_member(c, member, host, false, c->G);
}
extern "C" lhmm_status lhmm_closure_set_gemm(lhmm_closure_t c, int path) {
  if (!c || (path != 0 && path != 1)) return LHMM_ERR_ARG;
  c->gemm_path = path;
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_closure_sync(lhmm_closure_t c) {
  if (!c) return LHMM_ERR_ARG;
  LHMM_CK(cudaDeviceSynchronize());
  int flag = 0;
  LHMM_CK(cudaMemcpy(&flag, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    LHMM_CK(cudaMemset(c->tc_err, 0, sizeof(int)));
    return LHMM_ERR_TIMEOUT;
  }
  return LHMM_OK;
}

extern "C" lhmm_status lhmm_closure_info(lhmm_closure_t c, int64_t* n_params_per_member,
                                         int64_t* steps) {
  if (!c) return LHMM_ERR_ARG;
  long long n = 0;
  for (int l = 0; l < c->n_layers; ++l) {
    const int O = (l == c->n_layers - 1) ? c->out_dim : c->hidden;
    const int I = (l == 0) ? c->in_dim : c->hidden;
    n += static_cast<long long>(O) * I + O;
  }
  if (n_params_per_member) *n_params_per_member = n;
  if (steps) *steps = c->step;
  return LHMM_OK;
}
