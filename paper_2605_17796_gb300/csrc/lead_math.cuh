// Device arithmetic shared by the statically compiled kernels and the min-sum kernel that the
// library specialises at run time (NVRTC). Self-contained: no includes, so NVRTC can compile it.
#pragma once

#ifndef LEAD_CHECKED
#define LEAD_CHECKED 0
#endif

namespace lead {

// Bounds test of a table-driven index (checked builds): true when 0 <= i < n; otherwise the
// first failure is recorded in rec = {failures, site, index, bound} and the caller skips the
// access. Release builds compile it to `true`.
__device__ __forceinline__ bool in_bounds(unsigned long long* rec, long long i, long long n, unsigned int site) {
#if LEAD_CHECKED
  if (i >= 0 && i < n) return true;
  if (rec && atomicAdd(rec, 1ull) == 0ull) {
    rec[1] = site;
    rec[2] = (unsigned long long)i;
    rec[3] = (unsigned long long)n;
  }
  return false;
#else
  (void)rec;
  (void)i;
  (void)n;
  (void)site;
  return true;
#endif
}

// m_l-bit field starting at bit `pos` of a packed bit row (the local syndrome s_v).
__device__ __forceinline__ unsigned int bit_field(const unsigned int* row, int pos, int len) {
  const int w = pos >> 5, sh = pos & 31;
  const unsigned int lo = row[w];
  const unsigned int hi = (sh + len > 32) ? row[w + 1] : 0u;
  const unsigned int v = __funnelshift_r(lo, hi, sh);
  return v & ((1u << len) - 1u);
}

// Prior LLR lambda(p) = ln((1 - p)/p) on the binary32 decision track, by linear interpolation in
// a table over p in [2^-23, 1/2]: node i is the binary32 number with bit pattern
// (i + 13312) << 16 (exponent and top 7 fraction bits of p), t0[i] = lambda at the node, t1[i] =
// slope to the next node; lambda = t0[i] + (p - node) * t1[i] (the difference is exact), and
// lambda(p) = -lambda(1 - p) for p > 1/2 (1 - p is exact there). Interpolation error ~8e-6.
constexpr int kLlrNode0 = 13312;
constexpr int kLlrNodes = 2817;

__device__ __forceinline__ float llr_interp(float p, const float* __restrict__ t0,
                                            const float* __restrict__ t1) {
  p = fminf(fmaxf(p, __uint_as_float(0x34000000u)), __uint_as_float(0x3F7FFFFEu));  // [2^-23, 1-2^-23]
  const bool hi = p > 0.5f;
  const float q = hi ? __fsub_rn(1.0f, p) : p;
  const unsigned int qb = __float_as_uint(q);
  const int i = (int)(qb >> 16) - kLlrNode0;
  const float d = __fsub_rn(q, __uint_as_float(qb & 0xFFFF0000u));
  const float lam = __fadd_rn(__ldg(t0 + i), __fmul_rn(d, __ldg(t1 + i)));
  return hi ? -lam : lam;
}

// The same interpolation with the (node value, slope) pairs interleaved in shared memory.
__device__ __forceinline__ float llr_interp_s(float p, const float2* tv) {
  p = fminf(fmaxf(p, __uint_as_float(0x34000000u)), __uint_as_float(0x3F7FFFFEu));
  const bool hi = p > 0.5f;
  const float q = hi ? __fsub_rn(1.0f, p) : p;
  const unsigned int qb = __float_as_uint(q);
  const int i = (int)(qb >> 16) - kLlrNode0;
  const float d = __fsub_rn(q, __uint_as_float(qb & 0xFFFF0000u));
  const float2 t = tv[i];
  const float lam = __fadd_rn(t.x, __fmul_rn(d, t.y));
  return hi ? -lam : lam;
}

__device__ __forceinline__ float merged_llr_s(float q0, float q1, float alpha, const float2* tv) {
  float h = __fadd_rn(q0, q1);
  h = __fmul_rn(h, 0.5f);
  return llr_interp_s(__fmul_rn(h, alpha), tv);
}

// Phase 2 and the prior LLR: p = alpha * ((q0 + q1) * 1/2) in binary32, then lambda(p).
__device__ __forceinline__ float merged_llr(float q0, float q1, float alpha, const float* __restrict__ t0,
                                            const float* __restrict__ t1) {
  float h = __fadd_rn(q0, q1);
  h = __fmul_rn(h, 0.5f);
  return llr_interp(__fmul_rn(h, alpha), t0, t1);
}

// The standalone baseline's prior: lambda of the binary32 rounding of the channel marginal p.
__device__ __forceinline__ float channel_llr(double p, const float* __restrict__ t0,
                                             const float* __restrict__ t1) {
  return llr_interp(__double2float_rn(p), t0, t1);
}

// ln x for positive normal binary64 x, evaluated with explicit round-to-nearest operations:
// x = 2^e m with m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh z, z = (m - 1)/(m + 1), the inverse
// hyperbolic tangent series (Abramowitz & Stegun 4.1.27) through z^25; coefficients 2/k are
// binary64 quotients. Used to build the lambda table.
__device__ __forceinline__ double log_series_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  long long e = (long long)((b >> 52) & 0x7FFull) - 1023;
  double m = __longlong_as_double((long long)((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
  if (m > __longlong_as_double(0x3FF6A09E667F3BCDll)) {   // sqrt 2
    m = __dmul_rn(m, 0.5);
    e += 1;
  }
  const double z = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double w = __dmul_rn(z, z);
  double s = __ddiv_rn(2.0, 25.0);
  for (int k = 23; k >= 1; k -= 2) s = __dadd_rn(__dmul_rn(s, w), __ddiv_rn(2.0, (double)k));
  return __dadd_rn(__dmul_rn((double)e, __longlong_as_double(0x3FE62E42FEFA39EFll)), __dmul_rn(z, s));
}

}  // namespace lead
