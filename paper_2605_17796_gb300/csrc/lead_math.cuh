// Device arithmetic shared by the statically compiled kernels and the min-sum kernel that the
// library specialises at run time (NVRTC). Its one include, lead_llr.cuh, is itself
// self-contained; the run-time kernel source concatenates both files (without the include line).
#pragma once

#include "lead_llr.cuh"

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

// The standalone baseline's prior: lambda of the channel marginal p (binary32, as the host
// passes it).
__device__ __forceinline__ float channel_llr(float p) { return llr_f32(p); }

}  // namespace lead
