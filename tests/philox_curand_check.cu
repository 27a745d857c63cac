// Test harness: the library's device Philox4x32-10 and Box-Muller next to
// cuRAND's Philox4x32-10 on the same (counter, key) pairs.  Built and loaded
// by tests/test_gpu_philox_curand.py; not part of the library.
#include <curand_kernel.h>

#include "lhmm_common.cuh"

namespace {

__global__ void philox_words(const uint4* ctr, const uint2* key, int n, uint2* mine, uint4* ref,
                             float* theta) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint4 c = ctr[t];
  const uint2 k = key[t];
  const uint2 w = lhmm::philox4x32_10_xy(c.x, c.y, c.z, c.w, k.x, k.y);
  mine[t] = w;
  ref[t] = curand_Philox4x32_10(c, k);
  theta[t] = lhmm::gauss_from_words(w.x, w.y);
}

}  // namespace

// ctr: n x 4 words, key: n x 2 words (host); mine: n x 2, ref: n x 4 words,
// theta: n floats (host).  Returns 0, or the CUDA error code.
extern "C" int philox_curand_check(const unsigned* ctr, const unsigned* key, int n, unsigned* mine,
                                   unsigned* ref, float* theta) {
  if (n <= 0) return 0;
  uint4 *d_ctr = nullptr, *d_ref = nullptr;
  uint2 *d_key = nullptr, *d_mine = nullptr;
  float* d_theta = nullptr;
  cudaError_t e = cudaMalloc(&d_ctr, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_ref, sizeof(uint4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_key, sizeof(uint2) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_mine, sizeof(uint2) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d_theta, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMemcpy(d_ctr, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_key, key, sizeof(uint2) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    philox_words<<<(n + 255) / 256, 256>>>(d_ctr, d_key, n, d_mine, d_ref, d_theta);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(mine, d_mine, sizeof(uint2) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ref, d_ref, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(theta, d_theta, sizeof(float) * n, cudaMemcpyDeviceToHost);
  cudaFree(d_ctr);
  cudaFree(d_ref);
  cudaFree(d_key);
  cudaFree(d_mine);
  cudaFree(d_theta);
  return static_cast<int>(e);
}
