// Device arithmetic shared by the statically compiled kernels and the min-sum kernel that the
// library specialises at run time (NVRTC). Self-contained: no includes, so NVRTC can compile it.
#pragma once

namespace lead {

// m_l-bit field starting at bit `pos` of a packed bit row (the local syndrome s_v).
__device__ __forceinline__ unsigned int bit_field(const unsigned int* row, int pos, int len) {
  const int w = pos >> 5, sh = pos & 31;
  const unsigned int lo = row[w];
  const unsigned int hi = (sh + len > 32) ? row[w + 1] : 0u;
  const unsigned int v = __funnelshift_r(lo, hi, sh);
  return v & ((1u << len) - 1u);
}

// Natural logarithm of a positive normal binary32 value, evaluated in binary32 with explicit
// round-to-nearest operations: x = 2^e m with m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh z with
// z = (m - 1)/(m + 1), the inverse-hyperbolic-tangent series (Abramowitz & Stegun 4.1.27)
// truncated after z^11; coefficients are the nearest binary32 values of 2/k.
__device__ __forceinline__ float log_series_f32(float x) {
  const unsigned int b = __float_as_uint(x);
  int e = (int)((b >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
  if (m > __uint_as_float(0x3FB504F3u)) {          // sqrt 2
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float z = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float w = __fmul_rn(z, z);
  float s = __uint_as_float(0x3E3A2E8Cu);                         // 2/11
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

// The standalone baseline's prior: the channel LLR ln((1 - p)/p) of the binary32 rounding of p.
__device__ __forceinline__ float channel_llr(double p) {
  float pf = __double2float_rn(p);
  pf = fminf(fmaxf(pf, __uint_as_float(0x34000000u)), __uint_as_float(0x3F7FFFFEu));
  return log_series_f32(__fdiv_rn(__fsub_rn(1.0f, pf), pf));
}

}  // namespace lead
