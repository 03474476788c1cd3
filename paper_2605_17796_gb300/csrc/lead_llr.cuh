// Prior LLR lambda(p) = ln((1 - p)/p) in binary32 arithmetic, accurate to about 2^-45 relative
// before its final rounding, so the result is the binary32 rounding of the exact value except
// when that value lies within the error of a rounding boundary (the library's exhaustive test
// counts those inputs). Self-contained (no includes): also compiled at run time by NVRTC.
//
// Method: double-float arithmetic (a value is hi + lo with |lo| <= ulp(hi)/2) with the
// error-free transformations TwoSum (Knuth, TAOCP vol. 2, sec. 4.2.2), Fast2Sum (Dekker 1971)
// and the exact product error fma(a, b, -ab); the logarithm by argument reduction
// x = 2^e m, m in [sqrt(1/2), sqrt(2)), and ln m = 2 artanh z = 2 (z + z^3/3 + z^5/5 + ...) with
// z = (m - 1)/(m + 1), |z| <= 0.1716 (Abramowitz & Stegun 4.1.27).
#pragma once

#ifndef LEAD_HD
#define LEAD_HD __host__ __device__ __forceinline__
#endif

namespace lead {
namespace dfl {

// IEEE binary32 operations with round-to-nearest and no contraction into fused multiply-adds
// (the device intrinsics; host builds of this header compile plain operations with
// -ffp-contract=off and fmaf).
LEAD_HD float add(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
LEAD_HD float sub(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
LEAD_HD float mul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
LEAD_HD float fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}
LEAD_HD float div(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fdiv_rn(a, b);
#else
  return a / b;
#endif
}
LEAD_HD float from_bits(unsigned int u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  __builtin_memcpy(&f, &u, 4);
  return f;
#endif
}
LEAD_HD unsigned int to_bits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  unsigned int u;
  __builtin_memcpy(&u, &f, 4);
  return u;
#endif
}

struct df {
  float hi, lo;
};

// a + b exactly (any magnitudes)
LEAD_HD df two_sum(float a, float b) {
  const float s = add(a, b);
  const float bb = sub(s, a);
  return {s, add(sub(a, sub(s, bb)), sub(b, bb))};
}
// a + b exactly, for |a| >= |b| (or a = 0)
LEAD_HD df fast_two_sum(float a, float b) {
  const float s = add(a, b);
  return {s, sub(b, sub(s, a))};
}
// a * b exactly
LEAD_HD df two_prod(float a, float b) {
  const float p = mul(a, b);
  return {p, fma(a, b, -p)};
}
LEAD_HD df add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  const df t = two_sum(x.lo, y.lo);
  s = fast_two_sum(s.hi, add(s.lo, t.hi));
  return fast_two_sum(s.hi, add(s.lo, t.lo));
}
LEAD_HD df mul(df x, df y) {
  const df p = two_prod(x.hi, y.hi);
  return fast_two_sum(p.hi, add(p.lo, fma(x.hi, y.lo, mul(x.lo, y.hi))));
}
LEAD_HD df mul(df x, float y) {
  const df p = two_prod(x.hi, y);
  return fast_two_sum(p.hi, fma(x.lo, y, p.lo));
}
// x / y: three quotient digits, each corrected by the remainder computed in double-float
LEAD_HD df div(df x, df y) {
  const float ry = div(1.0f, y.hi);
  const float q1 = mul(x.hi, ry);
  df r = add(x, mul(y, -q1));
  const float q2 = mul(r.hi, ry);
  r = add(r, mul(y, -q2));
  const float q3 = mul(r.hi, ry);
  return add(fast_two_sum(q1, q2), df{q3, 0.0f});
}

// hi + lo splits of the constants; each part is a binary64 value rounded once to binary32
#define LEAD_DF_CONST(v) df{(float)(v), (float)((v) - (double)(float)(v))}

}  // namespace dfl

// lambda(p) = ln((1 - p)/p) for binary32 p, clamped to [2^-23, 1 - 2^-23]. For p > 1/2 the value
// is -lambda(1 - p) (1 - p is exact there), so the function is odd about 1/2 and lambda(1/2) = 0.
LEAD_HD float llr_f32(float p) {
  using namespace dfl;
  p = fminf(fmaxf(p, from_bits(0x34000000u)), from_bits(0x3F7FFFFEu));   // [2^-23, 1 - 2^-23]
  const bool neg = p > 0.5f;
  if (neg) p = sub(1.0f, p);
  // x = (1 - p)/p >= 1 as a double-float; 1 - p exactly by TwoSum
  const df x = div(two_sum(1.0f, -p), df{p, 0.0f});
  // x = 2^e m with m in [sqrt(1/2), sqrt(2)): exponent and significand of x.hi, scaled exactly
  const unsigned int b = to_bits(x.hi);
  int e = (int)((b >> 23) & 0xFFu) - 127;
  unsigned int mb = (b & 0x007FFFFFu) | 0x3F800000u;
  if (mb > 0x3FB504F3u) {          // significand above sqrt(2) (0x3FB504F3 = binary32 below it)
    mb -= 0x00800000u;
    e += 1;
  }
  const float scale = from_bits((unsigned int)(127 - e) << 23);    // 2^-e, e in [0, 24]
  const df m{from_bits(mb), mul(x.lo, scale)};
  // z = (m - 1)/(m + 1); m.hi - 1 is exact (Sterbenz)
  const df num = two_sum(sub(m.hi, 1.0f), m.lo);
  df den = two_sum(m.hi, 1.0f);
  den = fast_two_sum(den.hi, add(den.lo, m.lo));
  const df z = div(num, den);
  const df w = mul(z, z);
  // ln m = 2z (1 + w/3 + w^2/5 + ...): the tail from w^4/9 on in binary32 (it is below 8.3e-8),
  // the first three coefficients in double-float
  float t = (float)(1.0 / 21.0);
  t = fma(t, w.hi, (float)(1.0 / 19.0));
  t = fma(t, w.hi, (float)(1.0 / 17.0));
  t = fma(t, w.hi, (float)(1.0 / 15.0));
  t = fma(t, w.hi, (float)(1.0 / 13.0));
  t = fma(t, w.hi, (float)(1.0 / 11.0));
  t = fma(t, w.hi, (float)(1.0 / 9.0));
  df u = add(LEAD_DF_CONST(1.0 / 7.0), mul(w, t));
  u = add(LEAD_DF_CONST(1.0 / 5.0), mul(w, u));
  u = add(LEAD_DF_CONST(1.0 / 3.0), mul(w, u));
  const df z2{mul(z.hi, 2.0f), mul(z.lo, 2.0f)};
  const df lnm = add(z2, mul(z2, mul(w, u)));
  // lambda = e ln 2 + ln m
  const df lam = add(mul(LEAD_DF_CONST(0.6931471805599453), (float)e), lnm);
  const float r = add(lam.hi, lam.lo);
  return neg ? -r : r;
}

// Phase 2 and the prior LLR: p = alpha * ((q0 + q1) * 1/2) in binary32, then lambda(p).
LEAD_HD float merged_llr(float q0, float q1, float alpha) {
  const float h = dfl::mul(dfl::add(q0, q1), 0.5f);
  return llr_f32(dfl::mul(h, alpha));
}

}  // namespace lead
