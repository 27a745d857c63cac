// lhmm_common.cuh -- device helpers shared by the LHMM kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lhmm.h"

#define LHMM_CK(call)                                    \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return lhmm_cuda_error(e_);   \
  } while (0)

lhmm_status lhmm_cuda_error(cudaError_t e);

namespace lhmm {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with Weyl-sequence key increments.  Returns the first
// two output words, the only ones the pair noise uses.
__device__ __forceinline__ uint2 philox4x32_10_xy(uint32_t c0, uint32_t c1, uint32_t c2,
                                                  uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint2(c0, c1);
}

// Standard normal from two words: u = (k + 1/2) 2^-23 with k the top 23 bits
// (exact in FP32, u in (0, 1)), then Box-Muller r cos(2 pi u2) with
// r = sqrt(-2 ln u1).  ln u1 uses the hardware log2 for u1 <= 3/4 and above it
// the series ln u = 2 artanh(z) = 2 (z + z^3/3 + z^5/5 + z^7/7 + z^9/9) with
// z = (u - 1)/(u + 1) in (-1/7, 0] (truncation below 4e-10 relative), so
// -2 ln u1 keeps its relative precision as u1 -> 1 where the hardware log2
// only has an absolute bound.  The hardware cosine is accurate on [-pi, pi],
// hence cos(2 pi u2) = -cos(2 pi (u2 - 1/2)).
__device__ __forceinline__ float gauss_from_words(uint32_t x0, uint32_t x1) {
  const float u1 = (static_cast<float>(x0 >> 9) + 0.5f) * 0x1p-23f;
  const float u2 = (static_cast<float>(x1 >> 9) + 0.5f) * 0x1p-23f;
  const float z = __fdividef(u1 - 1.f, u1 + 1.f);
  const float z2 = z * z;
  const float poly =
      fmaf(z2, fmaf(z2, fmaf(z2, fmaf(z2, 1.f / 9.f, 1.f / 7.f), 1.f / 5.f), 1.f / 3.f), 1.f);
  const float ln_u1 = u1 > 0.75f ? 2.f * z * poly : __log2f(u1) * 0.693147181f;
  const float s = -2.f * ln_u1;  // >= 1.19e-7: u1 <= 1 - 2^-24
  return -(s * rsqrtf(s)) * __cosf(6.283185307f * (u2 - 0.5f));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace lhmm
