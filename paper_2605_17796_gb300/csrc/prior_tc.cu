// Phase 1 with per-qubit priors (Algorithm 1, LocalDecoder under a product prior) with its two
// contractions on the tensor cores (tcgen05).
//
// For one item (shot, vertex) the exact local posterior groups the local coset by row images:
// row a of the Delta x Delta view takes a pattern x of Delta bits; its image f = R_B x is one of
// NF = 2^kB classes; R_a(f) = log2 of the summed weights of the class's patterns (weights
// relative to the all-zero pattern, prior LLRs lambda_ab = ln((1-p)/p)); the row images F of the
// coset are F_i = base(s) + kern_i, i < NK; L_i = sum_a R_a(f_a(F_i)); and
//   q_ab = sum_i 2^{L_i} rho_ab(f_a(F_i)) / sum_i 2^{L_i},  rho_ab(f) = the class's share with x_b = 1.
// Writing f_a(F_i) = f_a(base) + k_a(i) turns both sums over the coset into products with the
// fixed 0/1 incidence matrix P[i][(a, g)] = [k_a(i) = g]:
//   GEMM1  L = R' P^T    R'[item][(a, g)] = R_a(g + f_a(base)) - max_f R_a(f)   (K = Delta NF)
//   GEMM2  A = W P       W[item][i] = 2^{L_i - max}                              (K = NK)
// and agg[a][f] = A[(a, f + f_a(base))] is the weight of the members whose row a lies in class f.
// A tile is 128 items = the MMA's M = the tensor-memory lanes. R' is split into two binary16
// terms (22 significant bits; the exact 0/1 incidence makes each product exact) and W into two
// bfloat16 terms (16 significant bits over binary32's exponent range), with binary32
// accumulation in tensor memory. The coset is taken in chunks of up to 128 members (GEMM1's N)
// that all add into one accumulator. The normaliser is the score of the least-cost member: a
// class's log-sum exceeds its best pattern's log-weight by at most log2 of the class size, and
// the least-cost member takes the best pattern of every row, so no member's score exceeds it by
// more than Delta log2(2^Delta / 2^kB) (18 for Delta = 6): every W is at most 2^18, and the
// least-cost member's own W is 1.
//
// On the CUDA cores: the prior LLRs, the class log-sums and shares (log-sum-exp in binary32),
// the least-cost local decision (exact integer costs W_ab = rint(2^20 lambda_ab), ties to the
// least row-major key, as the CUDA-core kernel and the oracle), the exponentials, and the
// marginals. Two threads share an item: thread `half` takes rows half*Delta/2 .. and half the
// members of the least-cost search.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "lead_device.cuh"
#include "tc_ptx.cuh"

namespace lead {
namespace {

constexpr int kTcThreads = 256;     // 8 warps: two threads per item
constexpr int kTile = 128;          // items per tile = MMA M = tensor-memory lanes
constexpr int kWaitPolls = 1 << 22; // bound of every wait on a tensor-core completion
constexpr float kLog2e = 1.4426950408889634f;

template <int DELTA, int KB, int NK>
struct TcShape {
  static constexpr int NL = DELTA * DELTA;
  static constexpr int NX = 1 << DELTA;           // row patterns
  static constexpr int NF = 1 << KB;              // row classes
  static constexpr int CS = NX / NF;              // patterns per class
  static constexpr int K1 = DELTA * NF;           // (row, class) pairs: GEMM1 depth, GEMM2 width
  static constexpr int CH = NK < 128 ? NK : 128;  // coset members per chunk (GEMM1 N, GEMM2 depth)
  static constexpr int NCH = NK / CH;
  static constexpr int HC = CH >= 32 ? 2 : 1;     // threads per item row in the chunk epilogue
  static constexpr int CW = CH / HC;              // members per thread in the chunk epilogue
  static constexpr int RH = DELTA / 2;            // rows per thread
  static constexpr int MPT = NK / 2;              // members per thread in the least-cost search
  // tensor memory: the chunk's scores in [0, CH), the accumulator at AGG0
  static constexpr int AGG0 = CH < 32 ? 32 : CH;
  static constexpr int TM_USED = AGG0 + (K1 < 32 ? 32 : 64);
  static constexpr int TM_COLS = TM_USED <= 32 ? 32 : TM_USED <= 64 ? 64 : TM_USED <= 128 ? 128
                                 : TM_USED <= 256 ? 256 : 512;
  static constexpr int CSTR = K1 + 1;             // int32 words per item in the cost table
  static constexpr int XSTR = K1 + 4;             // bytes per item in the pattern table
  // shared memory (bytes)
  static constexpr size_t B1 = 0;                                  // NK x K1 binary16 (GEMM1 B)
  static constexpr size_t B2 = B1 + (size_t)NK * K1 * 2;           // K1 x NK bfloat16 (GEMM2 B)
  static constexpr size_t A1 = B2 + (size_t)K1 * NK * 2;           // 2 terms x 128 x K1 binary16
  static constexpr size_t A1_TERM = (size_t)kTile * K1 * 2;
  static constexpr size_t A2 = A1 + 2 * A1_TERM;                   // 2 terms x 128 x CH bfloat16
  static constexpr size_t A2_TERM = (size_t)kTile * CH * 2;
  static constexpr size_t SCRATCH = (size_t)kTcThreads * NX * 4;   // per-thread pattern weights
  static constexpr size_t A2_BYTES = 2 * A2_TERM > SCRATCH ? 2 * A2_TERM : SCRATCH;
  static constexpr size_t COST = A2 + A2_BYTES;                    // 128 x CSTR int32
  static constexpr size_t XMIN = COST + (size_t)kTile * CSTR * 4;  // 128 x XSTR uint8
  static constexpr size_t KERN = (XMIN + (size_t)kTile * XSTR + 15) & ~size_t(15);   // NK uint32
  static constexpr size_t BEST = KERN + (size_t)NK * 4;            // 2 x 128 (cost, member) int2
  static constexpr size_t XCLS = BEST + 2 * (size_t)kTile * 8;     // NX uint8
  static constexpr size_t BYTES = (XCLS + NX + 15) & ~size_t(15);
  static_assert(BYTES <= 227 * 1024, "shared memory of one CTA");
  static_assert(CH % 16 == 0 && K1 % 16 == 0 && CW % 16 == 0, "MMA shapes");
  static_assert(DELTA % 2 == 0, "two threads per item split the rows");
};

struct TcArgs {
  int n, order, words_m;
  int64_t items;                // shots x order
  const uint32_t* syn;
  const float* lam;             // shots x n prior LLRs lambda(p)
  const uint16_t* views;
  const uint8_t* xcls;          // row patterns, class-major, increasing within a class
  const uint32_t* cbase;        // 2^m_l packed row images with R_A F = S
  const uint32_t* ckern;        // NK packed row images with R_A F = 0, increasing
  float* Q;                     // items x nl boosted local posteriors
  unsigned long long* ml;       // items: least-cost local decision (bit j = local index j), or null
  unsigned int* err;            // bit 0: a wait on the tensor cores ran out
};

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
  return (uint32_t)__half_as_ushort(__float2half_rn(lo)) | ((uint32_t)__half_as_ushort(__float2half_rn(hi)) << 16);
}
__device__ __forceinline__ uint32_t pack_bf162(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

// This thread's pattern-weight scratch: x at (x ^ lane) so that a pattern every lane reads at once
// falls in 32 different banks.
template <int NX>
__device__ __forceinline__ int scr_index(int tid, int x) {
  return tid * NX + (x ^ ((tid & 31) & (NX - 1)));
}

// 2^x by the hardware's approximate base-2 exponential (ex2.approx.ftz, relative error about
// 2^-22; results below 2^-126 flush to 0, far below every sum they enter here).
__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// v[g] <- v[g ^ p] for a runtime p in [0, N): one conditional swap stage per bit of p, so the
// array stays in registers.
template <int N>
__device__ __forceinline__ void xor_permute(float (&v)[N], uint32_t p) {
#pragma unroll
  for (int bit = 1; bit < N; bit <<= 1) {
    const bool sw = (p & (uint32_t)bit) != 0;
#pragma unroll
    for (int g = 0; g < N; ++g) {
      if (g & bit) continue;
      const float x = v[g], y = v[g | bit];
      v[g] = sw ? y : x;
      v[g | bit] = sw ? x : y;
    }
  }
}

__host__ __device__ constexpr int lowest_bit(int x) { return (x & 1) ? 0 : 1 + lowest_bit(x >> 1); }

// log2-weights of the 2^Delta patterns of one row relative to the all-zero pattern, into scratch:
// l(x) = l(x without its lowest bit) - w_lowest.
template <int DELTA>
__device__ __forceinline__ void row_weights(float* scr, int tid, const float (&w)[DELTA]) {
  constexpr int NX = 1 << DELTA;
  float l[NX];
  l[0] = 0.0f;
#pragma unroll
  for (int x = 1; x < NX; ++x) {
    const int low = lowest_bit(x);
    l[x] = l[x & (x - 1)] - w[low];
  }
#pragma unroll
  for (int x = 0; x < NX; ++x) scr[scr_index<NX>(tid, x)] = l[x];
}

// Integer costs of the 2^Delta patterns of one row (sum of the costs of its set bits), into the
// same scratch as row_weights, as int bit patterns: c(x) = c(x without its lowest bit) + W_lowest.
template <int DELTA>
__device__ __forceinline__ void row_costs(float* scr, int tid, const int (&W)[DELTA]) {
  constexpr int NX = 1 << DELTA;
  int c[NX];
  c[0] = 0;
#pragma unroll
  for (int x = 1; x < NX; ++x) c[x] = c[x & (x - 1)] + W[lowest_bit(x)];
#pragma unroll
  for (int x = 0; x < NX; ++x) scr[scr_index<NX>(tid, x)] = __int_as_float(c[x]);
}

template <int DELTA, int KB, int ML, int NK>
__global__ void __launch_bounds__(kTcThreads, 1) prior_local_tc_kernel(TcArgs a) {
  using S = TcShape<DELTA, KB, NK>;
  constexpr int NL = S::NL, NX = S::NX, NF = S::NF, CS = S::CS, K1 = S::K1, CH = S::CH, CW = S::CW;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar_g1, mbar_g2;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = (warp & 3) * 32 + lane;         // item row of the tile = tensor-memory lane
  const int half = warp >> 2;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  uint32_t* kern_s = reinterpret_cast<uint32_t*>(sm + S::KERN);
  uint8_t* xcls_s = sm + S::XCLS;
  float* scr = reinterpret_cast<float*>(sm + S::A2);
  int* cost_s = reinterpret_cast<int*>(sm + S::COST);
  uint8_t* xmin_s = sm + S::XMIN;
  int2* best_s = reinterpret_cast<int2*>(sm + S::BEST);

  // ---- once per CTA: coset tables and the two incidence operands (exact 0/1) ----
  for (int i = tid; i < NK; i += kTcThreads) kern_s[i] = __ldg(a.ckern + i);
  for (int i = tid; i < NX; i += kTcThreads) xcls_s[i] = __ldg(a.xcls + i);
  for (int e = tid; e < NK * K1; e += kTcThreads) {
    const int m = e / K1, k = e - m * K1;
    const int ra = k / NF, g = k - ra * NF;
    const bool one = ((__ldg(a.ckern + m) >> (ra * KB)) & (NF - 1)) == (uint32_t)g;
    *reinterpret_cast<uint16_t*>(sm + S::B1 + tc::kmajor_offset(m, k, NK)) = one ? 0x3C00u : 0u;   // 1.0 in binary16
    *reinterpret_cast<uint16_t*>(sm + S::B2 + tc::kmajor_offset(k, m, K1)) = one ? 0x3F80u : 0u;   // 1.0 in bfloat16
  }
  if (tid == 0) {
    tc::mbar_init(&mbar_g1, 1);
    tc::mbar_init(&mbar_g2, 1);
    tc::mbar_init_fence();
    abort_s = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base_s, S::TM_COLS);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base_s;
  const uint32_t idesc1 = tc::idesc_f16(kTile, CH, false);
  const uint32_t idesc2 = tc::idesc_f16(kTile, K1, true);
  uint32_t ph_g1 = 0, ph_g2 = 0;          // parity of the next phase of each barrier

  // GEMM1 of chunk c: scores[item][member] for the members c*CH .. c*CH + CH - 1 (two terms of R')
  auto issue_gemm1 = [&](int c) {
    const uint32_t a1 = tc::smem_addr(sm + S::A1), b1 = tc::smem_addr(sm + S::B1);
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int ks = 0; ks < K1 / 16; ++ks) {
        const uint64_t ad = tc::smem_desc(a1 + (uint32_t)(t * S::A1_TERM) + (uint32_t)(ks * 2 * kTile * 16), kTile * 16, 128);
        const uint64_t bd = tc::smem_desc(b1 + (uint32_t)((c * CH / 8) * 128) + (uint32_t)(ks * 2 * NK * 16), NK * 16, 128);
        tc::mma_f16(tbase, ad, bd, idesc1, t > 0 || ks > 0);
      }
  };
  // GEMM2 of chunk c: acc[item][(a, g)] += the chunk's W times the incidence (two terms of W)
  auto issue_gemm2 = [&](int c) {
    const uint32_t a2 = tc::smem_addr(sm + S::A2), b2 = tc::smem_addr(sm + S::B2);
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int ks = 0; ks < CH / 16; ++ks) {
        const uint64_t ad = tc::smem_desc(a2 + (uint32_t)(t * S::A2_TERM) + (uint32_t)(ks * 2 * kTile * 16), kTile * 16, 128);
        const uint64_t bd = tc::smem_desc(b2 + (uint32_t)(((c * CH + ks * 16) / 8) * (K1 * 16)), K1 * 16, 128);
        tc::mma_f16(tbase + (uint32_t)S::AGG0, ad, bd, idesc2, c > 0 || t > 0 || ks > 0);
      }
  };
  auto wait_or_abort = [&](uint64_t* mbar, uint32_t& ph) {
    if (!tc::mbar_wait(mbar, ph, kWaitPolls)) {
      abort_s = 1;
      if (a.err) atomicOr(a.err, 1u);
    }
    ph ^= 1u;
  };
  // key of coset member i for this item: the least-cost pattern of every row, row a at bit a*Delta
  auto key_of = [&](int i) {
    const uint32_t k = kern_s[i];
    const uint8_t* xrow = xmin_s + row * S::XSTR;
    unsigned long long key = 0;
#pragma unroll
    for (int ra = 0; ra < DELTA; ++ra)
      key |= (unsigned long long)xrow[ra * NF + ((k >> (ra * KB)) & (NF - 1))] << (ra * DELTA);
    return key;
  };

  const int64_t ntiles = (a.items + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t item = tile * kTile + row;
    const bool active = item < a.items;
    const int64_t shot = active ? item / a.order : 0;
    const int v = active ? (int)(item - shot * a.order) : 0;
    const uint32_t s = active ? bit_field(a.syn + shot * a.words_m, v * ML, ML) : 0u;
    const uint32_t fb = __ldg(a.cbase + s);
    const float* lam_row = a.lam + shot * a.n;
    const uint16_t* vrow = a.views + v * NL;

    // ---- this thread's rows: prior LLRs (log2 units), integer costs, class log-sums, least-cost
    // patterns; the R' operand (two binary16 terms) and the permuted cost / pattern tables ----
#pragma unroll 1
    for (int rr = 0; rr < S::RH; ++rr) {
      const int ra = half * S::RH + rr;
      float wl[DELTA];
      int Wc[DELTA];
#pragma unroll
      for (int b = 0; b < DELTA; ++b) {
        const float lam = active ? __ldg(lam_row + __ldg(vrow + b * DELTA + ra)) : 0.0f;
        wl[b] = lam * kLog2e;
        Wc[b] = __float2int_rn(__fmul_rn(lam, 1048576.0f));
      }
      row_weights<DELTA>(scr, tid, wl);
      const uint32_t fba = (fb >> (ra * KB)) & (NF - 1);
      float R[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        float m = -INFINITY, lx[CS];
#pragma unroll
        for (int t = 0; t < CS; ++t) {
          lx[t] = scr[scr_index<NX>(tid, xcls_s[f * CS + t])];
          m = fmaxf(m, lx[t]);
        }
        float sum = 0.0f;
#pragma unroll
        for (int t = 0; t < CS; ++t) sum += fast_exp2(lx[t] - m);
        R[f] = m + __log2f(sum);
      }
      // least-cost pattern of every class (the class lists patterns in increasing order, so the
      // first least cost is the least pattern)
      row_costs<DELTA>(scr, tid, Wc);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        int cmin = INT_MAX, xmin = 0;
#pragma unroll
        for (int t = 0; t < CS; ++t) {
          const int x = xcls_s[f * CS + t];
          const int c = __float_as_int(scr[scr_index<NX>(tid, x)]);
          if (c < cmin) {
            cmin = c;
            xmin = x;
          }
        }
        const int g = f ^ (int)fba;
        cost_s[row * S::CSTR + ra * NF + g] = cmin;
        xmin_s[row * S::XSTR + ra * NF + g] = (uint8_t)xmin;
      }
      float rmax = -INFINITY;
#pragma unroll
      for (int f = 0; f < NF; ++f) rmax = fmaxf(rmax, R[f]);
      xor_permute<NF>(R, fba);            // R[g] = log-sum of class g ^ fba
      // R'[(ra, g)] = R[g] - rmax as two binary16 terms, NF consecutive K columns
      uint32_t hi[NF / 2], lo[NF / 2];
#pragma unroll
      for (int g = 0; g < NF; g += 2) {
        const float v0 = active ? R[g] - rmax : 0.0f, v1 = active ? R[g + 1] - rmax : 0.0f;
        const float h0 = __half2float(__float2half_rn(v0)), h1 = __half2float(__float2half_rn(v1));
        hi[g / 2] = pack_half2(v0, v1);
        lo[g / 2] = pack_half2(v0 - h0, v1 - h1);
      }
      unsigned char* p0 = sm + S::A1 + tc::kmajor_offset(row, ra * NF, kTile);
      if constexpr (NF == 8) {
        *reinterpret_cast<uint4*>(p0) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(p0 + S::A1_TERM) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      } else {
        *reinterpret_cast<uint2*>(p0) = make_uint2(hi[0], hi[1]);
        *reinterpret_cast<uint2*>(p0 + S::A1_TERM) = make_uint2(lo[0], lo[1]);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (abort_s) break;
    if (tid == 0) {
      tc::fence_after_sync();
      issue_gemm1(0);
      tc::mma_commit(&mbar_g1);
    }

    // ---- least-cost local decision over this thread's half of the coset (overlaps the MMAs) ----
    {
      int best = INT_MAX, bi = half * S::MPT;
      const int* crow = cost_s + row * S::CSTR;
#pragma unroll 2
      for (int i0 = 0; i0 < S::MPT; ++i0) {
        const int i = half * S::MPT + i0;
        const uint32_t k = kern_s[i];
        int c = 0;
#pragma unroll
        for (int ra = 0; ra < DELTA; ++ra) c += crow[ra * NF + ((k >> (ra * KB)) & (NF - 1))];
        if (c < best) {
          best = c;
          bi = i;
        } else if (c == best && key_of(i) < key_of(bi)) {
          bi = i;
        }
      }
      best_s[half * kTile + row] = make_int2(best, bi);
    }
    __syncthreads();
    // the least-cost member over both halves: (cost, key), lexicographic; its score (from the R'
    // operand, as the tensor cores see it) is the normaliser of W
    int ml_member;
    {
      const int2 b0 = best_s[row], b1 = best_s[kTile + row];
      const bool second = b1.x < b0.x || (b1.x == b0.x && key_of(b1.y) < key_of(b0.y));
      ml_member = second ? b1.y : b0.y;
    }
    float M = 0.0f;
    {
      const uint32_t k = kern_s[ml_member];
#pragma unroll
      for (int ra = 0; ra < DELTA; ++ra) {
        const uint32_t off = tc::kmajor_offset(row, ra * NF + (int)((k >> (ra * KB)) & (NF - 1)), kTile);
        M += __half2float(__ushort_as_half(*reinterpret_cast<const uint16_t*>(sm + S::A1 + off))) +
             __half2float(__ushort_as_half(*reinterpret_cast<const uint16_t*>(sm + S::A1 + S::A1_TERM + off)));
      }
    }

    // ---- chunks: scores -> W = 2^(score - M) (two bfloat16 terms) -> GEMM2 ----
#pragma unroll 1
    for (int c = 0; c < S::NCH; ++c) {
      wait_or_abort(&mbar_g1, ph_g1);
      if (c > 0) wait_or_abort(&mbar_g2, ph_g2);   // the previous GEMM2 has read A2
      tc::fence_after_sync();
      const bool mine = S::HC == 2 || half == 0;
      const int col0 = S::HC == 2 ? half * CW : 0;
      if (mine && !abort_s) {
#pragma unroll
        for (int j = 0; j < CW; j += 16) {
          float sc[16];
          tc::tmem_ld16(tbase + lane_base + (uint32_t)(col0 + j), sc);
#pragma unroll
          for (int h8 = 0; h8 < 16; h8 += 8) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
              const float w0 = fast_exp2(sc[h8 + u] - M), w1 = fast_exp2(sc[h8 + u + 1] - M);
              const float g0 = __bfloat162float(__float2bfloat16_rn(w0));
              const float g1 = __bfloat162float(__float2bfloat16_rn(w1));
              hi[u / 2] = pack_bf162(w0, w1);
              lo[u / 2] = pack_bf162(w0 - g0, w1 - g1);
            }
            unsigned char* p0 = sm + S::A2 + tc::kmajor_offset(row, col0 + j + h8, kTile);
            *reinterpret_cast<uint4*>(p0) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(p0 + S::A2_TERM) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();                     // scores of the chunk read, its W in place
      if (abort_s) break;
      if (tid == 0) {
        tc::fence_after_sync();
        issue_gemm2(c);
        tc::mma_commit(&mbar_g2);
        if (c + 1 < S::NCH) {
          issue_gemm1(c + 1);
          tc::mma_commit(&mbar_g1);
        }
      }
    }
    if (abort_s) break;
    wait_or_abort(&mbar_g2, ph_g2);
    tc::fence_after_sync();
    __syncthreads();
    if (abort_s) break;

    // ---- marginals, boost, store ----
    unsigned long long mask = 0;
    {
      const unsigned long long key = key_of(ml_member);
#pragma unroll
      for (int ra = 0; ra < DELTA; ++ra)
#pragma unroll
        for (int b = 0; b < DELTA; ++b) mask |= ((key >> (ra * DELTA + b)) & 1ull) << (b * DELTA + ra);
    }
    float rz = 0.0f;
#pragma unroll 1
    for (int rr = 0; rr < S::RH; ++rr) {
      const int ra = half * S::RH + rr;
      float wl[DELTA];
#pragma unroll
      for (int b = 0; b < DELTA; ++b)
        wl[b] = (active ? __ldg(lam_row + __ldg(vrow + b * DELTA + ra)) : 0.0f) * kLog2e;
      row_weights<DELTA>(scr, tid, wl);
      const uint32_t fba = (fb >> (ra * KB)) & (NF - 1);
      float agg[NF];
      {
        float t16[16];
        tc::tmem_ld16(tbase + lane_base + (uint32_t)(S::AGG0 + (ra * NF) / 16 * 16), t16);
        const int off = (ra * NF) % 16;    // the row's NF columns within the 16 loaded
#pragma unroll
        for (int g = 0; g < NF; ++g) {
          agg[g] = t16[g];
#pragma unroll
          for (int o = NF; o < 16; o += NF)
            if (off == o) agg[g] = t16[o + g];
        }
      }
      if (rr == 0) {                       // every row's classes partition the coset: Z
        float Z = 0.0f;
#pragma unroll
        for (int g = 0; g < NF; ++g) Z += agg[g];
        rz = 1.0f / Z;
      }
      xor_permute<NF>(agg, fba);           // agg[f] = weight of the members whose row ra is in class f
      // every pattern's share of its class, times the class's weight, in place of its log-weight
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        float m = -INFINITY, ex[CS];
#pragma unroll
        for (int t = 0; t < CS; ++t) {
          ex[t] = scr[scr_index<NX>(tid, xcls_s[f * CS + t])];
          m = fmaxf(m, ex[t]);
        }
        float sum = 0.0f;
#pragma unroll
        for (int t = 0; t < CS; ++t) {
          ex[t] = fast_exp2(ex[t] - m);
          sum += ex[t];
        }
        const float wgt = agg[f] / sum;
#pragma unroll
        for (int t = 0; t < CS; ++t) scr[scr_index<NX>(tid, xcls_s[f * CS + t])] = wgt * ex[t];
      }
      // q_b (times Z) = the weighted shares of the patterns with bit b set
      float qb[DELTA];
#pragma unroll
      for (int b = 0; b < DELTA; ++b) qb[b] = 0.0f;
#pragma unroll
      for (int x = 1; x < NX; ++x) {
        const float u = scr[scr_index<NX>(tid, x)];
#pragma unroll
        for (int b = 0; b < DELTA; ++b)
          if ((x >> b) & 1) qb[b] += u;
      }
      if (active) {
#pragma unroll
        for (int b = 0; b < DELTA; ++b) {
          const int j = b * DELTA + ra;
          float q = qb[b] * rz;
          if ((mask >> j) & 1ull) q = fmaxf(q, 0.5f);
          a.Q[item * NL + j] = q;
        }
      }
    }
    if (active && half == 0 && a.ml) a.ml[item] = mask;
    __syncthreads();                       // scratch, tables and A1 are rewritten by the next tile
  }
  // every MMA this CTA issued has completed (each commit was waited for, or the wait ran out)
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tbase, S::TM_COLS);
}

template <int DELTA, int KB, int ML, int NK>
int launch_tc(const lead_code* code, int side, const uint32_t* syn, int64_t shots, const float* lam, float* Q,
              uint64_t* ml, unsigned int* err, cudaStream_t stream) {
  using S = TcShape<DELTA, KB, NK>;
  const DeviceSide& ds = code->dside[side];
  TcArgs a{};
  a.n = code->n;
  a.order = code->order;
  a.words_m = code->side[side].params.words_m;
  a.items = shots * code->order;
  a.syn = syn;
  a.lam = lam;
  a.views = ds.views;
  a.xcls = ds.xcls;
  a.cbase = ds.cbase;
  a.ckern = ds.ckern;
  a.Q = Q;
  a.ml = reinterpret_cast<unsigned long long*>(ml);
  a.err = err;
  auto kern = prior_local_tc_kernel<DELTA, KB, ML, NK>;
  LEAD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::BYTES));
  const int64_t tiles = (a.items + kTile - 1) / kTile;
  const int64_t blocks = std::min<int64_t>(tiles, (int64_t)sm_count(code->device));
  kern<<<(unsigned)blocks, kTcThreads, S::BYTES, stream>>>(a);
  LEAD_CUDA_TRY(cudaGetLastError());
  return LEAD_OK;
}

}  // namespace

// Phase 1 with per-qubit priors on the tensor cores: lam (shots x n, the prior LLRs lambda(p))
// -> Q (shots x order x nl boosted posteriors), ml (nullable). Local codes (Delta, k_B, m_l, NK)
// = (6, 3, 9, 512) and (4, 2, 4, 16); others give LEAD_EINVAL.
int run_prior_local_tc(const lead_code* code, int side, const uint32_t* syn, int64_t shots, const float* lam,
                       float* Q, uint64_t* ml, unsigned int* err, cudaStream_t stream) {
  const HostSide& hs = code->side[side];
  const DeviceSide& ds = code->dside[side];
  if (!ds.xcls || !ds.cbase || !ds.ckern) return LEAD_EINVAL;
  const size_t nk = hs.ckern.size();
  if (code->delta == 6 && hs.kRB == 3 && hs.m_l == 9 && nk == 512)
    return launch_tc<6, 3, 9, 512>(code, side, syn, shots, lam, Q, ml, err, stream);
  if (code->delta == 4 && hs.kRB == 2 && hs.m_l == 4 && nk == 16)
    return launch_tc<4, 2, 4, 16>(code, side, syn, shots, lam, Q, ml, err, stream);
  return LEAD_EINVAL;
}

}  // namespace lead
