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

// e^x for binary64 x in [-88, 88]: Cody-Waite reduction k = rint(x / ln 2), r = (x - k LN2_HI) -
// k LN2_LO with the fdlibm split of ln 2 (LN2_HI has 21 trailing zero bits, so k LN2_HI is exact),
// e^r by its Taylor series through r^14 in Horner form, times 2^k (exact). Separate
// round-to-nearest binary64 operations throughout.
__device__ __forceinline__ double exp_series_f64(double x) {
  const double kInvLn2 = __longlong_as_double(0x3FF71547652B82FEll);
  const double kLn2Hi = __longlong_as_double(0x3FE62E42FEE00000ll);
  const double kLn2Lo = __longlong_as_double(0x3DEA39EF35793C76ll);
  constexpr double kInvFact[15] = {1.0 / 1.0, 1.0 / 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0,
                                   1.0 / 720.0, 1.0 / 5040.0, 1.0 / 40320.0, 1.0 / 362880.0,
                                   1.0 / 3628800.0, 1.0 / 39916800.0, 1.0 / 479001600.0,
                                   1.0 / 6227020800.0, 1.0 / 87178291200.0};
  const double k = rint(__dmul_rn(x, kInvLn2));
  const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(k, kLn2Hi)), __dmul_rn(k, kLn2Lo));
  double s = kInvFact[14];
  for (int n = 13; n >= 0; --n) s = __dadd_rn(__dmul_rn(s, r), kInvFact[n]);
  return ldexp(s, (int)k);
}

// q = 1 / (1 + e^post) in binary32 from a binary32 posterior LLR (clamped to [-88, 88]).
__device__ __forceinline__ float sigmoid_f32(float post) {
  const double x = (double)fminf(fmaxf(post, -88.0f), 88.0f);
  return __double2float_rn(__ddiv_rn(1.0, __dadd_rn(1.0, exp_series_f64(x))));
}

int sm_count(int device);

// Class tables of a local posterior table, laid out in the `extra` workspace part that follows
// the table (local_pair_extra_bytes): the class byte of every entry, header[0] = K (0 when the
// table has more distinct values than a byte holds) and the K x K pair table.
struct ClassTables {
  uint8_t* cls;
  int* header;
  unsigned int* pair;
};
ClassTables class_tables(const lead_code* code, int side, void* extra);
size_t local_pair_extra_bytes(const lead_code* code, int side);
// Builds them on `stream` for alpha; pair entries in the storage format of `prec`.
int launch_classify(const lead_code* code, int side, float alpha, int prec, const float* table, void* extra,
                    cudaStream_t stream);

// min(cap, remaining) for the shot loops of the persistent kernels.
__host__ __device__ __forceinline__ int rows_left(int64_t cap, int64_t remaining) {
  return (int)(remaining < cap ? remaining : cap);
}

}  // namespace lead
