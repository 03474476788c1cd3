// Device helpers shared by the LEAD kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lead_internal.h"

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

// m_l-bit field starting at bit `pos` of a packed bit row (the local syndrome s_v).
__device__ __forceinline__ uint32_t bit_field(const uint32_t* row, int pos, int len) {
  const int w = pos >> 5, sh = pos & 31;
  uint32_t lo = row[w];
  uint32_t hi = (sh + len > 32) ? row[w + 1] : 0u;
  uint32_t v = __funnelshift_r(lo, hi, sh);
  return v & ((1u << len) - 1u);
}

// Natural logarithm of a positive normal binary32 value, evaluated in binary32 with explicit
// round-to-nearest operations: x = 2^e m with m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh z with
// z = (m - 1)/(m + 1), the inverse-hyperbolic-tangent series (Abramowitz & Stegun 4.1.27)
// truncated after z^11; coefficients are the nearest binary32 values of 2/k.
__device__ __forceinline__ float log_series_f32(float x) {
  const uint32_t b = __float_as_uint(x);
  int e = (int)((b >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
  if (m > __uint_as_float(0x3FB504F3u)) {          // sqrt 2
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float z = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float w = __fmul_rn(z, z);
  float s = __uint_as_float(0x3E3A2E8Cu);          // 2/11
  s = __fadd_rn(__fmul_rn(s, w), __uint_as_float(0x3E638E39u));   // 2/9
  s = __fadd_rn(__fmul_rn(s, w), __uint_as_float(0x3E924925u));   // 2/7
  s = __fadd_rn(__fmul_rn(s, w), __uint_as_float(0x3ECCCCCDu));   // 2/5
  s = __fadd_rn(__fmul_rn(s, w), __uint_as_float(0x3F2AAAABu));   // 2/3
  s = __fadd_rn(__fmul_rn(s, w), 2.0f);                            // 2/1
  const float a = __fmul_rn((float)e, __uint_as_float(0x3F317218u));  // e ln 2
  return __fadd_rn(a, __fmul_rn(z, s));
}

// Phase 2 and the prior LLR: p = alpha * ((q0 + q1) * 1/2), clamped to [2^-23, 1 - 2^-23],
// lambda = ln((1 - p)/p), all in binary32 round-to-nearest.
__device__ __forceinline__ float merged_llr(float q0, float q1, float alpha) {
  float h = __fadd_rn(q0, q1);
  h = __fmul_rn(h, 0.5f);
  float p = __fmul_rn(h, alpha);
  p = fminf(fmaxf(p, __uint_as_float(0x34000000u)), __uint_as_float(0x3F7FFFFEu));
  return log_series_f32(__fdiv_rn(__fsub_rn(1.0f, p), p));
}

__device__ __forceinline__ float channel_llr(double p) {
  float pf = __double2float_rn(p);
  pf = fminf(fmaxf(pf, __uint_as_float(0x34000000u)), __uint_as_float(0x3F7FFFFEu));
  return log_series_f32(__fdiv_rn(__fsub_rn(1.0f, pf), pf));
}

int sm_count(int device);

// min(cap, remaining) for the shot loops of the persistent kernels.
__host__ __device__ __forceinline__ int rows_left(int64_t cap, int64_t remaining) {
  return (int)(remaining < cap ? remaining : cap);
}

}  // namespace lead
