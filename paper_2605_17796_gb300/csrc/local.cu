// Phases 1-2 as a standalone kernel (lead_local_estimate) by class and pair tables.
//
// For a given side, p and alpha, the boosted local posterior q(s, j) takes few distinct values
// (40 for the Delta = 6 codes, 3 for Delta = 4): the coset weight enumerators of a local code
// repeat across syndromes and positions. The prior LLR of a qubit is a function of the two
// values its views see, lambda(alpha * ((q0 + q1) * 1/2)), so it is tabulated once per call over
// the K x K pairs of distinct values, with the same binary32 arithmetic as the direct
// evaluation (the results are bit-identical). Per (shot, qubit) the kernel then does two class
// lookups and one pair lookup instead of two table lookups, the merge and the logarithm.
//
//   classify_kernel   one CTA: the distinct values of the table (a hash set in shared memory),
//                     ranked by value (class ids are deterministic), the class byte of every
//                     table entry, and the K x K pair table in the output format;
//   local_pair_kernel the per-(shot, qubit) lookups; when K exceeds the shared pair capacity it
//                     evaluates the merge directly instead (uniform branch).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "lead_device.cuh"

namespace lead {

namespace {

constexpr int kHashSlots = 512;        // open addressing over the float bit patterns
constexpr int kMaxClasses = 255;       // class ids fit a byte
constexpr int kPairSmem = 64;          // pair tables of up to 64 x 64 entries are staged in shared memory
constexpr unsigned int kEmpty = 0xFFFFFFFFu;   // a NaN pattern; q is never NaN
constexpr int kClassThreads = 1024;

// The stored pattern of an LLR in the precision mode's format (round to nearest even; binary16
// saturating at +-65504).
template <int PREC>
__device__ __forceinline__ unsigned int llr_bits(float v) {
  if constexpr (PREC == LEAD_PREC_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  else if constexpr (PREC == LEAD_PREC_FP16)
    return __half_as_ushort(__float2half_rn(fminf(fmaxf(v, -65504.0f), 65504.0f)));
  else return __float_as_uint(v);
}

__device__ __forceinline__ unsigned int hash_slot(unsigned int key) {
  return (key * 2654435761u) >> 23;    // 9 bits: Knuth's multiplicative hash
}

// Probe for key; inserts it when absent. Returns the slot, or -1 when the set is full.
__device__ __forceinline__ int find_or_insert(unsigned int* keys, unsigned int key) {
  unsigned int h = hash_slot(key);
  for (int probe = 0; probe < kHashSlots; ++probe) {
    const unsigned int prev = atomicCAS(keys + h, kEmpty, key);
    if (prev == kEmpty || prev == key) return (int)h;
    h = (h + 1) & (kHashSlots - 1);
  }
  return -1;
}

struct ClassArgs {
  const float* table;     // T boosted local posteriors
  int T;
  float alpha;
  uint8_t* cls;           // T class ids
  int* header;            // [0] = K (0: more than kMaxClasses distinct values)
  unsigned int* pair;     // K x K stored LLR patterns (float bits or 16-bit patterns)
};

template <int PREC>
__global__ void __launch_bounds__(kClassThreads) classify_kernel(ClassArgs a) {
  __shared__ unsigned int keys[kHashSlots];
  __shared__ int rank_of[kHashSlots];
  __shared__ float vals[kMaxClasses];
  __shared__ int full, count;
  const int tid = threadIdx.x;
  for (int i = tid; i < kHashSlots; i += blockDim.x) keys[i] = kEmpty;
  if (tid == 0) {
    full = 0;
    count = 0;
  }
  __syncthreads();
  for (int e = tid; e < a.T; e += blockDim.x)
    if (find_or_insert(keys, __float_as_uint(__ldg(a.table + e))) < 0) full = 1;
  __syncthreads();
  // rank of every occupied slot among the occupied ones (q >= 0: bit order = value order)
  for (int i = tid; i < kHashSlots; i += blockDim.x) {
    const unsigned int k = keys[i];
    int r = -1;
    if (k != kEmpty) {
      r = 0;
      for (int j = 0; j < kHashSlots; ++j) r += (keys[j] != kEmpty && keys[j] < k) ? 1 : 0;
      atomicAdd(&count, 1);
    }
    rank_of[i] = r;
  }
  __syncthreads();
  const int K = (full || count > kMaxClasses) ? 0 : count;
  if (K == 0) {
    if (tid == 0) a.header[0] = 0;
    return;
  }
  for (int i = tid; i < kHashSlots; i += blockDim.x)
    if (rank_of[i] >= 0) vals[rank_of[i]] = __uint_as_float(keys[i]);
  __syncthreads();
  for (int e = tid; e < a.T; e += blockDim.x)
    a.cls[e] = (uint8_t)rank_of[find_or_insert(keys, __float_as_uint(__ldg(a.table + e)))];
  for (int idx = tid; idx < K * K; idx += blockDim.x) {
    const int c0 = idx / K, c1 = idx - c0 * K;
    a.pair[idx] = llr_bits<PREC>(merged_llr(vals[c0], vals[c1], a.alpha));
  }
  if (tid == 0) a.header[0] = K;
}

constexpr int kPairThreads = 512;
constexpr int kPairShotBatch = 32;

struct PairArgs {
  int n, order, words_m, m_l, T;
  float alpha;
  int64_t shots;
  const uint32_t* syn;
  const uint8_t* cls;
  const unsigned int* pair;
  const int* header;
  const float* table;           // direct evaluation when the pair table does not fit
  const uint32_t* qslots;
  void* llr;                    // float, or the 16-bit pattern of the storage format
  unsigned long long* check;    // checked build: bounds-failure record
};

// Staged local syndromes are vertex-major: sv_s[v * kSvStride + shot]; the padded row of 36
// 16-bit entries (72 bytes) spreads consecutive vertices over the banks, and four shots of one
// vertex come with one 8-byte load.
constexpr int kSvStride = 36;
static_assert(kPairShotBatch % 4 == 0 && kPairShotBatch <= kSvStride && (kSvStride * 2) % 8 == 0,
              "four-shot loads stay inside an 8-byte-aligned row");

// The shots of one staged batch: every thread takes qubits tid, tid + blockDim, ... and for
// each produces its LLR in every shot of the batch (consecutive threads on consecutive qubits,
// so each store is coalesced; the shots give independent lookups to overlap). FAST: class and
// pair lookups; otherwise the direct merge from the posterior table.
template <int NL, int PREC, bool FAST, typename OutT>
__device__ __forceinline__ void batch_llrs(const PairArgs& a, const uint16_t* sv_s, const uint8_t* cls_s,
                                           const OutT* pair_s, int K, int64_t b0, int nsh, OutT* out) {
  for (int i = threadIdx.x; i < a.n; i += kPairThreads) {
    const uint32_t s0 = __ldg(a.qslots + 2 * i), s1 = __ldg(a.qslots + 2 * i + 1);
    if (!in_bounds(a.check, s0, (long long)a.order * NL, 10) || !in_bounds(a.check, s1, (long long)a.order * NL, 10))
      continue;
    const uint16_t* p0 = sv_s + (s0 / NL) * kSvStride;
    const uint16_t* p1 = sv_s + (s1 / NL) * kSvStride;
    const int j0 = (int)(s0 % NL), j1 = (int)(s1 % NL);
    OutT* o = out + b0 * (int64_t)a.n + i;
    for (int sl = 0; sl < nsh; sl += 4) {
      const uint2 w0 = *reinterpret_cast<const uint2*>(p0 + sl);
      const uint2 w1 = *reinterpret_cast<const uint2*>(p1 + sl);
      const uint32_t a0[4] = {w0.x & 0xFFFFu, w0.x >> 16, w0.y & 0xFFFFu, w0.y >> 16};
      const uint32_t a1[4] = {w1.x & 0xFFFFu, w1.x >> 16, w1.y & 0xFFFFu, w1.y >> 16};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (sl + u < nsh) {
          const int e0 = (int)a0[u] * NL + j0;
          const int e1 = (int)a1[u] * NL + j1;
          OutT v;
          if constexpr (FAST) {
            const int c0 = cls_s[e0], c1 = cls_s[e1];
            v = (in_bounds(a.check, c0, K, 11) && in_bounds(a.check, c1, K, 11)) ? pair_s[c0 * K + c1] : OutT(0);
          } else {
            const float x = merged_llr(__ldg(a.table + e0), __ldg(a.table + e1), a.alpha);
            if constexpr (PREC == LEAD_PREC_FP32) v = x;
            else v = (unsigned short)llr_bits<PREC>(x);
          }
          __stcs(o + (sl + u) * (int64_t)a.n, v);
        }
      }
    }
  }
}

// Per batch of 32 shots the local syndromes of all vertices are extracted once into shared
// memory, then batch_llrs runs over the batch. Entries of shots past the batch's end are read
// (in bounds) and never used.
template <int NL, int PREC>
__global__ void __launch_bounds__(kPairThreads, 3) local_pair_kernel(PairArgs a) {
  using OutT = typename std::conditional<PREC == LEAD_PREC_FP32, float, unsigned short>::type;
  extern __shared__ __align__(16) unsigned char sm[];
  const int cls_bytes = (a.T + 15) & ~15;
  uint8_t* cls_s = sm;
  OutT* pair_s = reinterpret_cast<OutT*>(sm + cls_bytes);
  uint16_t* sv_s = reinterpret_cast<uint16_t*>(sm + cls_bytes + kPairSmem * kPairSmem * sizeof(OutT));
  const int K = __ldg(a.header);
  const bool fast = K > 0 && K <= kPairSmem;     // uniform across the grid
  if (fast) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(a.cls);
    uint32_t* dst = reinterpret_cast<uint32_t*>(cls_s);
    for (int i = threadIdx.x; i < a.T / 4; i += blockDim.x) dst[i] = __ldg(src + i);
    for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
      const unsigned int bits = __ldg(a.pair + i);
      if constexpr (PREC == LEAD_PREC_FP32) pair_s[i] = __uint_as_float(bits);
      else pair_s[i] = (unsigned short)bits;
    }
  }
  const int wm = a.words_m, V = a.order, ml = a.m_l;
  OutT* out = static_cast<OutT*>(a.llr);
  for (int64_t b0 = (int64_t)blockIdx.x * kPairShotBatch; b0 < a.shots; b0 += (int64_t)gridDim.x * kPairShotBatch) {
    const int nsh = rows_left(kPairShotBatch, a.shots - b0);
    __syncthreads();
    for (int i = threadIdx.x; i < nsh * V; i += blockDim.x) {
      const int sl = i / V, v = i - sl * V;
      sv_s[v * kSvStride + sl] = (uint16_t)bit_field(a.syn + (b0 + sl) * wm, v * ml, ml);
    }
    __syncthreads();
    if (fast) batch_llrs<NL, PREC, true>(a, sv_s, cls_s, pair_s, K, b0, nsh, out);
    else batch_llrs<NL, PREC, false>(a, sv_s, cls_s, pair_s, K, b0, nsh, out);
  }
}

}  // namespace

size_t local_pair_extra_bytes(const lead_code* code, int side) {
  const size_t T = (size_t)(1 << code->side[side].m_l) * code->nl;
  const size_t pair = ((size_t)kMaxClasses * kMaxClasses * 4 + 255) / 256 * 256;
  return (T + 255) / 256 * 256 + 256 + pair;     // a multiple of 256: callers may lay sides end to end
}

// Phases 1-2 through class and pair tables; `extra` (local_pair_extra_bytes, 16-byte aligned)
// holds the class bytes, the header and the pair table. Returns LEAD_EINVAL for local codes
// other than Delta = 4 or 6, or when the staged tables exceed one CTA's shared memory.
ClassTables class_tables(const lead_code* code, int side, void* extra) {
  const int T = (1 << code->side[side].params.m_l) * code->nl;
  ClassTables t;
  t.cls = static_cast<uint8_t*>(extra);
  t.header = reinterpret_cast<int*>(t.cls + (T + 255) / 256 * 256);
  t.pair = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(t.header) + 256);
  return t;
}

// The class bytes, K and the K x K pair table of a local posterior table, for alpha, with the pair
// entries stored in the format of `prec` (binary32 bits for LEAD_PREC_FP32).
int launch_classify(const lead_code* code, int side, float alpha, int prec, const float* table, void* extra,
                    cudaStream_t stream) {
  const int T = (1 << code->side[side].params.m_l) * code->nl;
  const ClassTables t = class_tables(code, side, extra);
  ClassArgs c{table, T, alpha, t.cls, t.header, t.pair};
  if (prec == LEAD_PREC_BF16) classify_kernel<LEAD_PREC_BF16><<<1, kClassThreads, 0, stream>>>(c);
  else if (prec == LEAD_PREC_FP16) classify_kernel<LEAD_PREC_FP16><<<1, kClassThreads, 0, stream>>>(c);
  else classify_kernel<LEAD_PREC_FP32><<<1, kClassThreads, 0, stream>>>(c);
  LEAD_CUDA_TRY(cudaGetLastError());
  return LEAD_OK;
}

int launch_local_pair(const lead_code* code, const lead_decode_opts* o, const uint32_t* syn, int64_t shots,
                      void* llr, const float* table, void* extra, cudaStream_t stream) {
  const SideParams& P = code->side[o->side].params;
  const int nl = code->nl;
  if (nl != 16 && nl != 36) return LEAD_EINVAL;
  const int T = (1 << P.m_l) * nl;
  const ClassTables ct = class_tables(code, o->side, extra);
  uint8_t* cls = ct.cls;
  int* header = ct.header;
  unsigned int* pair = ct.pair;
  int rc = launch_classify(code, o->side, o->alpha, o->precision, table, extra, stream);
  if (rc != LEAD_OK) return rc;

  PairArgs a{};
  a.n = code->n;
  a.order = code->order;
  a.words_m = P.words_m;
  a.m_l = P.m_l;
  a.T = T;
  a.alpha = o->alpha;
  a.shots = shots;
  a.syn = syn;
  a.cls = cls;
  a.pair = pair;
  a.header = header;
  a.table = table;
  a.qslots = code->dside[o->side].qslots;
  a.llr = llr;
  a.check = code->d_check;
  const size_t esize = o->precision == LEAD_PREC_FP32 ? 4 : 2;
  const size_t smem = (size_t)((T + 15) & ~15) + (size_t)kPairSmem * kPairSmem * esize +
                      sizeof(uint16_t) * (size_t)kSvStride * code->order;
  if (smem > 227u * 1024u) return LEAD_EINVAL;
  auto go = [&](auto kern) -> int {
    if (smem > 48 * 1024)
      LEAD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    LEAD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPairThreads, smem));
    per_sm = std::max(per_sm, 1);
    const int64_t batches = (shots + kPairShotBatch - 1) / kPairShotBatch;
    const int64_t blocks = std::min<int64_t>(batches, (int64_t)sm_count(code->device) * per_sm);
    kern<<<(unsigned)blocks, kPairThreads, smem, stream>>>(a);
    LEAD_CUDA_TRY(cudaGetLastError());
    return LEAD_OK;
  };
  auto by_prec = [&](auto nlc) -> int {
    constexpr int NLv = decltype(nlc)::value;
    if (o->precision == LEAD_PREC_BF16) return go(local_pair_kernel<NLv, LEAD_PREC_BF16>);
    if (o->precision == LEAD_PREC_FP16) return go(local_pair_kernel<NLv, LEAD_PREC_FP16>);
    return go(local_pair_kernel<NLv, LEAD_PREC_FP32>);
  };
  if (nl == 16) return by_prec(std::integral_constant<int, 16>{});
  return by_prec(std::integral_constant<int, 36>{});
}

}  // namespace lead
