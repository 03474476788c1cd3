// Device helpers shared by the LEAD kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lead_internal.h"
#include "lead_math.cuh"

#define LEAD_CUDA_TRY(expr)                      \
  do {                                           \
    cudaError_t _e = (expr);                     \
    if (_e != cudaSuccess) return LEAD_ECUDA;    \
  } while (0)

namespace lead {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of two 32x32->64 products of
// counter words 0 and 2 with M0 = 0xD2511F53 and M1 = 0xCD9E8D57, the halves permuted and XORed
// with the remaining words and the round key; the key advances by (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

int sm_count(int device);

// min(cap, remaining) for the shot loops of the persistent kernels.
__host__ __device__ __forceinline__ int rows_left(int64_t cap, int64_t remaining) {
  return (int)(remaining < cap ? remaining : cap);
}

}  // namespace lead
