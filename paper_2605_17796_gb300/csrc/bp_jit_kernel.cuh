// Global min-sum decoder (Phase 3 of Algorithm 1, with Phases 1-2 fused into its prologue),
// specialised at run time (NVRTC) to one code side. The generated prelude defines
//   LEAD_NL (Delta^2), LEAD_ML (local rows m_l), LEAD_TS (threads with work = shots per CTA *
//   |G|), LEAD_BLOCK (block size), LEAD_MINBLOCKS (CTAs per SM), LEAD_KMAX, LEAD_JMAX,
//   LEAD_PREC (storage format), and the constant tables lead_jit::kLen[ML] (row weights),
//   kSupp[ML][KMAX] (local indices of every local row, increasing), kRowLo[ML] / kRowHi[ML]
//   (the same rows as masks over the two hard-decision words) and, per slot j, kJLen[NL],
//   kJRow[NL][JMAX], kJPos[NL][JMAX] (the local rows touching j in increasing order and j's
//   position in each row's support),
// so every loop over a check's support below has compile-time trip counts and offsets.
//
// Mapping: one CTA handles `spb` shots; thread t = shot sl * |G| + vertex v. Shared memory is
// slot-major with row stride LEAD_TS: word j * TS + t belongs to local index j of thread t.
//   U[j][t]    sum of the messages of the vertex's local rows into its slot j,
//   post[j][t] posterior LLR of the slot,  lam[j][t] prior LLR of the slot.
// The global table pa[j][t] holds the shared-memory address of the partner slot (the qubit's
// other view) with bit 15 set when this view belongs to the smaller vertex. Each thread keeps
// the compressed state of its ML local checks in registers: (min1, min2, meta), meta bits 0..25
// = signs of the v2c messages by support position, the first position in the highest of the
// row's len bits (position k at bit len - 1 - k: each sign is shifted in from below), 26..30 =
// position of the first minimum, 31 = parity s_c + sum of signs. The message to position k is (-1)^(parity + sign_k) times
// (k == argmin ? min2 : min1), exactly the minimum over the other positions.
//
// Order of operations (identical to the oracle's binary32 decision track):
//   post_i = (lambda_i + U_v0) + U_v1 (v0 < v1 the qubit's two views), U_v accumulated from 0 in
//   increasing local row order; v2c = post - c2v_old; hard decision e_i = [post_i < 0];
//   iteration t tests H e = s first and stops at the first success (t = 0 tests the prior).

namespace lead_jit {
// Storage format of every LLR the decoder keeps between steps (LEAD_PREC: 0 binary32, 1 bfloat16,
// 2 binary16): the prior, the check-to-variable magnitudes, the per-vertex sums U and the
// posteriors. Arithmetic is binary32; a value is rounded to nearest even when stored (binary16
// saturates at +-65504: min-sum magnitudes can grow past its range over many iterations).
#if LEAD_PREC == 0
typedef float msg_t;
__device__ __forceinline__ msg_t enc(float v) { return v; }
__device__ __forceinline__ float dec(msg_t h) { return h; }
#else
typedef unsigned short msg_t;
__device__ __forceinline__ msg_t enc(float v) {
  unsigned short h;
#if LEAD_PREC == 1
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(v));
#else
  // saturating: magnitudes beyond the largest finite binary16 (65504) are stored as 65504
  v = fminf(fmaxf(v, -65504.0f), 65504.0f);
  asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(v));
#endif
  return h;
}
__device__ __forceinline__ float dec(msg_t h) {
#if LEAD_PREC == 1
  return __uint_as_float((unsigned int)h << 16);
#else
  float f;
  asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
  return f;
#endif
}
#endif
__device__ __forceinline__ float rnd(float v) { return dec(enc(v)); }

// Hard decisions of a thread's NL slots as two words, each decision shifted in from below with
// one funnel shift: slot j < 32 ends at bit min(NL, 32) - 1 - j of lo, slot j >= 32 at bit
// NL - 1 - j of hi (kRowLo / kRowHi hold the local rows in this layout).
struct HardBits {
  unsigned int lo = 0u, hi = 0u;
  // the decision [x < 0] of slot j (j in increasing order): x + 0 turns -0 into +0 and keeps
  // every other value, so its sign bit is the decision; the shift takes that bit alone
  __device__ __forceinline__ void push_neg(int j, float x) {
    const unsigned int w = __float_as_uint(__fadd_rn(x, 0.0f));
    if (j < 32) lo = __funnelshift_l(w, lo, 1);
    else hi = __funnelshift_l(w, hi, 1);
  }
  __device__ __forceinline__ bool get(int j) const {
    constexpr int nlo = LEAD_NL < 32 ? LEAD_NL : 32;
    return j < 32 ? (lo >> (nlo - 1 - j)) & 1u : (hi >> (LEAD_NL - 1 - j)) & 1u;
  }
  __device__ __forceinline__ unsigned int row_parity(int r) const {
    return (unsigned int)(__popc(lo & kRowLo[r]) + (LEAD_NL > 32 ? __popc(hi & kRowHi[r]) : 0)) & 1u;
  }
};

// The two stored magnitudes (min1, min2) of a local row's compressed state: two binary32
// registers, or both 16-bit patterns packed in one register.
struct RowMag {
#if LEAD_PREC == 0
  float a, b;
  __device__ __forceinline__ float m1() const { return a; }
  __device__ __forceinline__ float m2() const { return b; }
  __device__ __forceinline__ void set(float n1, float n2) {
    a = n1;
    b = n2;
  }
#else
  unsigned int w;
  __device__ __forceinline__ float m1() const { return dec((msg_t)(w & 0xFFFFu)); }
  __device__ __forceinline__ float m2() const { return dec((msg_t)(w >> 16)); }
  __device__ __forceinline__ void set(float n1, float n2) { w = (unsigned int)enc(n1) | ((unsigned int)enc(n2) << 16); }
#endif
};

// Shared-memory offset (bytes) of the word arrays behind the three NL x TS message arrays.
[[maybe_unused]] constexpr unsigned int kMsgBytes = ((3u * LEAD_NL * LEAD_TS * (unsigned int)sizeof(msg_t)) + 15u) & ~15u;

// Phases 1-2 for one slot: the merged prior LLR of the table entries e0 (this view) and e1 (the
// partner view), lambda(alpha * ((q(e0) + q(e1)) * 1/2)). With K > 0 classes it is one lookup in
// the K x K pair table the entry point built with the same arithmetic (bit-identical); otherwise
// the merge is evaluated here.
__device__ __forceinline__ float merged_prior(const lead::BPJitArgs& a, int K, int e0, int e1) {
  if (K > 0) {
    const int c0 = __ldg(a.cls + e0), c1 = __ldg(a.cls + e1);
    const bool ok = lead::in_bounds(a.check, c0, K, 5) && lead::in_bounds(a.check, c1, K, 5);
    return ok ? __ldg(a.pair + c0 * K + c1) : 0.0f;
  }
  return lead::merged_llr(__ldg(a.table + e0), __ldg(a.table + e1), a.alpha);
}

// New check-to-variable message of a local row of len positions to its k-th support position,
// from the row's compressed state (m1, m2 magnitudes; meta = signs | argmin << 26 | parity << 31).
__device__ __forceinline__ float c2v_msg(float m1, float m2, unsigned int meta, int k, int len) {
  const unsigned int flip = meta ^ (0u - (meta >> 31));   // bit len-1-k: sign of the message to k
  const float mag = (k == (int)((meta >> 26) & 31u)) ? m2 : m1;
  return __uint_as_float(__float_as_uint(mag) ^ (((flip >> (len - 1 - k)) & 1u) << 31));
}

// Check-node update of the thread's ML local rows (sv: their syndrome bits) from the posteriors
// of its own slots in P: every v2c = post - c2v_old, then the row's new (min1, min2, meta).
__device__ __forceinline__ void check_update(RowMag (&mag)[LEAD_ML], unsigned int (&meta)[LEAD_ML], unsigned int sv,
                                             const msg_t* P, int tid) {
#pragma unroll
  for (int r = 0; r < LEAD_ML; ++r) {
    const float m1o = mag[r].m1(), m2o = mag[r].m2();
    const unsigned int mo = meta[r];
    const int amo = (int)((mo >> 26) & 31u);
    const unsigned int flip = mo ^ (0u - (mo >> 31));   // bit len-1-k: sign of the old message to k
    float n1 = __int_as_float(0x7F800000), n2 = __int_as_float(0x7F800000);
    int am = 0;
    unsigned int sg = 0;
#pragma unroll
    for (int k = 0; k < LEAD_KMAX; ++k) {
      if (k >= kLen[r]) break;      // constant after unrolling
      const float mago = (k == amo) ? m2o : m1o;
      const float co = __uint_as_float(__float_as_uint(mago) ^ ((flip >> (kLen[r] - 1 - k)) << 31));
      const float v2c = __fsub_rn(dec(P[kSupp[r][k] * LEAD_TS + tid]), co);
      const float m = fabsf(v2c);
      // v2c is never -0 (every sum starts from +0 terms): its sign bit equals v2c < 0
      sg = __funnelshift_l(__float_as_uint(v2c), sg, 1);
      const bool lt = m < n1;
      n2 = lt ? n1 : fminf(n2, m);
      n1 = lt ? m : n1;
      am = lt ? k : am;
    }
    const unsigned int par = ((unsigned int)__popc(sg) ^ (sv >> r)) & 1u;
    mag[r].set(n1, n2);
    meta[r] = sg | ((unsigned int)am << 26) | (par << 31);
  }
}

// U of every slot from the rows' new states: the messages of the rows touching the slot summed
// in increasing row order (binary32, the first term stored as is: 0 + c == c), stored once into
// U (own slots).
__device__ __forceinline__ void store_u(const RowMag (&mag)[LEAD_ML], const unsigned int (&meta)[LEAD_ML], msg_t* U,
                                        int tid) {
#pragma unroll
  for (int j = 0; j < LEAD_NL; ++j) {
    float u = 0.0f;
#pragma unroll
    for (int i = 0; i < LEAD_JMAX; ++i) {
      if (i >= kJLen[j]) break;     // constant after unrolling
      const int r = kJRow[j][i];
      const float c = c2v_msg(mag[r].m1(), mag[r].m2(), meta[r], kJPos[j][i], kLen[r]);
      u = (i == 0) ? c : __fadd_rn(u, c);
    }
    U[j * LEAD_TS + tid] = enc(u);
  }
}

// Posterior of slot j from the prior lj, this view's sum uo and the partner view's sum up, in
// the qubit's order (lambda + U_first) + U_second.
__device__ __forceinline__ float slot_post(bool first, float lj, float uo, float up) {
  return first ? __fadd_rn(__fadd_rn(lj, uo), up) : __fadd_rn(__fadd_rn(lj, up), uo);
}
}  // namespace lead_jit

#if LEAD_CLUSTER == 1
namespace lead_jit {

// Iteration schedule. With one shot per CTA (LEAD_SPB == 1) an iteration has one barrier: the
// first two message arrays, X and Y, trade roles every iteration. Phase A reads the sums U of the previous
// iteration from X (own and partner slots) and writes the posteriors into Y; the check update
// reads the thread's own posteriors from Y and then overwrites them with the new sums U; the
// barrier (which also gathers the local check failures into the shot's verdict) orders those
// writes before the partners' reads in the next iteration, whose posteriors go into X. The
// verdict of iteration t is therefore known after its check update, which a converged shot
// computes once in vain; the outputs are the posteriors of iteration t, recomputed from X.
// With several shots per CTA each shot has its own verdict, and the iteration keeps two
// barriers (timed faster than one barrier with every thread reading every shot's verdict);
// a shot that has stopped leaves its threads idle until the batch is done.
extern "C" __global__ void __launch_bounds__(LEAD_BLOCK, LEAD_MINBLOCKS)
lead_bp_jit(const lead::BPJitArgs a) {
  constexpr int NL = LEAD_NL, ML = LEAD_ML, TS = LEAD_TS;
  extern __shared__ __align__(16) unsigned int smem[];
  const int V = a.order, spb = a.spb, wm = a.words_m;
  msg_t* Us = reinterpret_cast<msg_t*>(smem);
  msg_t* Ps = Us + NL * TS;
  msg_t* Ls = Ps + NL * TS;
#if LEAD_ALIAS
  // one shot per CTA: the staged syndromes live in the posterior array (read by the prologue
  // only, before the first iteration writes posteriors) and the correction bits in the array
  // whose sums U are dead when the shot stops
  unsigned int* syn_s = reinterpret_cast<unsigned int*>(Ps);
#else
  unsigned int* syn_s = smem + kMsgBytes / 4;
  unsigned int* cb = syn_s + spb * wm;
  int* flags = reinterpret_cast<int*>(cb + spb * a.words_n);     // per-shot verdicts (several shots)
  (void)flags;
#endif
  const unsigned short* __restrict__ PA = a.pa;

  const int tid = threadIdx.x;
  const int sl = tid / V, v = tid - sl * V;
  const bool lane_ok = tid < TS;
  const float lam_ch = a.use_lead ? 0.0f : lead::channel_llr(a.p);
  const int K = (a.use_lead && a.header) ? __ldg(a.header) : 0;   // classes of the local table

  for (long long g0 = (long long)blockIdx.x * spb; g0 < a.shots; g0 += (long long)gridDim.x * spb) {
    const int nsh = (int)((a.shots - g0) < spb ? (a.shots - g0) : spb);
    for (int i = tid; i < nsh * wm; i += blockDim.x) syn_s[i] = __ldg(a.syn + g0 * wm + i);
#if LEAD_SPB > 1
    for (int i = tid; i < spb * a.words_n; i += blockDim.x) cb[i] = 0u;
    if (tid < 2 * spb) flags[tid] = 0;
#endif
    __syncthreads();
    const bool act = lane_ok && sl < nsh;
    RowMag mag[ML];
    unsigned int meta[ML];
#pragma unroll
    for (int r = 0; r < ML; ++r) {
      mag[r].set(0.0f, 0.0f);
      meta[r] = 0u;
    }
    unsigned int sv = 0;
    if (act) {
      const unsigned int* srow = syn_s + sl * wm;
      sv = lead::bit_field(srow, v * ML, ML);
#pragma unroll 2
      for (int j = 0; j < NL; ++j) {
        float lj;
        if (a.lam) {
          const int q = __ldg(a.views + v * NL + j);
          lj = lead::in_bounds(a.check, q, a.n, 3) ? __ldg(a.lam + (g0 + sl) * a.n + q) : 0.0f;
        } else if (a.use_lead) {
          const unsigned int addr = __ldg(PA + j * TS + tid) & 0x7FFFu;
          const unsigned int jp = addr / TS, vp = addr - jp * TS - sl * V;
          const bool ok = lead::in_bounds(a.check, addr, NL * TS, 1) && lead::in_bounds(a.check, vp, V, 2);
          const unsigned int svp = ok ? lead::bit_field(srow, vp * ML, ML) : 0u;
          lj = merged_prior(a, K, sv * NL + j, svp * NL + jp);
        } else {
          lj = lam_ch;
        }
        Ls[j * TS + tid] = enc(lj);
        Us[j * TS + tid] = enc(0.0f);
      }
    }
    __syncthreads();
#if LEAD_SPB == 1
    msg_t* X = Us;      // sums U of the previous iteration
    msg_t* Y = Ps;      // this iteration's posteriors, then its sums U
    for (int t = 0;; ++t) {
      HardBits hm;
      unsigned int bad = 0;
      if (act) {
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const unsigned int pa = __ldg(PA + j * TS + tid);
          const float up = lead::in_bounds(a.check, pa & 0x7FFFu, NL * TS, 1) ? dec(X[pa & 0x7FFFu]) : 0.0f;
          const msg_t pe = enc(slot_post(pa >> 15, dec(Ls[j * TS + tid]), dec(X[j * TS + tid]), up));
          Y[j * TS + tid] = pe;
          hm.push_neg(j, dec(pe));
        }
#pragma unroll
        for (int r = 0; r < ML; ++r) bad |= (hm.row_parity(r) ^ (sv >> r)) & 1u;
      }
      const bool last = t >= a.max_iter;      // uniform
      if (act && !last) {
        check_update(mag, meta, sv, Y, tid);
        store_u(mag, meta, Y, tid);
      }
      // the block-wide OR of the local check failures is the shot's verdict
      const bool conv = !__syncthreads_or(bad);
      if (conv || last) {                      // uniform across the CTA
#if LEAD_ALIAS
        unsigned int* cbw = reinterpret_cast<unsigned int*>(Y);
#else
        unsigned int* cbw = cb;
#endif
        for (int i = tid; i < a.words_n; i += blockDim.x) cbw[i] = 0u;
        __syncthreads();
        if (act) {
          for (int j = 0; j < NL; ++j) {
            const unsigned int pa = __ldg(PA + j * TS + tid);
            if (pa >> 15) {
              const int q = __ldg(a.views + v * NL + j);
              if (!lead::in_bounds(a.check, q, a.n, 3)) continue;
              if (hm.get(j)) atomicOr(cbw + (q >> 5), 1u << (q & 31));
              if (a.llr) {
                // the posterior of iteration t again, from the same stored operands
                const float up = lead::in_bounds(a.check, pa & 0x7FFFu, NL * TS, 1) ? dec(X[pa & 0x7FFFu]) : 0.0f;
                a.llr[g0 * a.n + q] = rnd(slot_post(true, dec(Ls[j * TS + tid]), dec(X[j * TS + tid]), up));
              }
            }
          }
          if (v == 0) {
            a.status[g0] = conv ? (unsigned char)1 : (unsigned char)2;
            if (a.iters) a.iters[g0] = t;
          }
        }
        __syncthreads();     // every thread's correction bits are in cbw before the copy-out
        for (int i = tid; i < a.words_n; i += blockDim.x) a.corr[g0 * a.words_n + i] = cbw[i];
        __syncthreads();     // the copy-out has read cbw before the next shot stages its syndromes
        break;
      }
      msg_t* const T = X;
      X = Y;
      Y = T;
    }
#else
    // several shots per CTA, each with its own verdict: two barriers per iteration (the verdicts
    // of all shots are read between them, so every thread leaves the loop at the same iteration)
    bool mydone = !act;
    for (int t = 0;; ++t) {
      HardBits hm;
      unsigned int bad = 0;
      if (!mydone) {
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const unsigned int pa = __ldg(PA + j * TS + tid);
          const float up = lead::in_bounds(a.check, pa & 0x7FFFu, NL * TS, 1) ? dec(Us[pa & 0x7FFFu]) : 0.0f;
          const msg_t pe = enc(slot_post(pa >> 15, dec(Ls[j * TS + tid]), dec(Us[j * TS + tid]), up));
          Ps[j * TS + tid] = pe;
          hm.push_neg(j, dec(pe));
        }
#pragma unroll
        for (int r = 0; r < ML; ++r) bad |= (hm.row_parity(r) ^ (sv >> r)) & 1u;
      }
      if (bad) atomicOr(flags + (t & 1) * spb + sl, 1);
      if (tid < spb) flags[((t + 1) & 1) * spb + tid] = 0;
      __syncthreads();
      const bool conv = flags[(t & 1) * spb + sl] == 0;
      if (!mydone && (conv || t >= a.max_iter)) {
        const long long shot = g0 + sl;
        for (int j = 0; j < NL; ++j) {
          if (__ldg(PA + j * TS + tid) >> 15) {
            const int q = __ldg(a.views + v * NL + j);
            if (!lead::in_bounds(a.check, q, a.n, 3)) continue;
            if (hm.get(j)) atomicOr(cb + sl * a.words_n + (q >> 5), 1u << (q & 31));
            if (a.llr) a.llr[shot * a.n + q] = dec(Ps[j * TS + tid]);
          }
        }
        if (v == 0) {
          a.status[shot] = conv ? (unsigned char)1 : (unsigned char)2;
          if (a.iters) a.iters[shot] = t;
        }
        mydone = true;
      }
      if (!__syncthreads_or(!mydone)) break;
      if (!mydone) {
        check_update(mag, meta, sv, Ps, tid);
        store_u(mag, meta, Us, tid);
      }
      __syncthreads();
    }
    __syncthreads();     // every thread's correction bits are in cb before the copy-out
    for (int i = tid; i < nsh * a.words_n; i += blockDim.x) a.corr[g0 * a.words_n + i] = cb[i];
    __syncthreads();
#endif
  }
}

}  // namespace lead_jit
#endif

#if LEAD_CLUSTER > 1
// ---------------------------------------------------------------------------------------------
// The same decoder for codes whose per-shot state exceeds one CTA's shared memory: a cluster of
// LEAD_CLUSTER CTAs handles one shot, CTA rank r owning vertices r*TS .. r*TS + TS - 1 (TS =
// LEAD_TS). A partner slot owned by another CTA is read from that CTA's shared memory through
// the cluster's distributed shared memory (mapa to a generic address, then a plain load). The iteration's one
// synchronisation point is a cluster barrier; the shot's verdict is one flag word in rank 0,
// OR-ed by every thread with a violated local check and read back by all threads after the
// barrier, so every CTA of the cluster takes the same branch at every step.
// The partner table [j][v] (per global vertex v) holds the partner slot's word address inside
// its owner CTA, the owner's rank and whether this view belongs to the smaller vertex: u16
// entries address | rank << 13 | first << 15 when LEAD_PA16, else u32 entries address |
// rank << 16 | first << 31.
// ---------------------------------------------------------------------------------------------
namespace lead_jit {

__device__ __forceinline__ unsigned int cluster_rank() {
  unsigned int r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Generic address of the same shared-memory location in CTA `rank` of the cluster: ordinary
// loads through it reach that CTA's shared memory (distributed shared memory), and the compiler
// schedules them like any other load.
__device__ __forceinline__ const msg_t* map_rank_generic(const msg_t* p, unsigned int rank) {
  unsigned long long out;
  asm("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<unsigned long long>(p)), "r"(rank));
  return reinterpret_cast<const msg_t*>(out);
}

__device__ __forceinline__ unsigned int map_rank(const void* p, unsigned int rank) {
  const unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
  unsigned int out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(a), "r"(rank));
  return out;
}

constexpr int kPartnerGroup = 12;      // partner reads in flight per thread

// Partner of slot (j, v) from the cluster partner table: word address inside the owner CTA,
// owner rank, and whether v is the qubit's first (smaller) vertex.
struct Partner {
  unsigned int addr, rank;
  bool first;
};
__device__ __forceinline__ Partner cluster_partner(const void* table, int j, int v, int V) {
  Partner p;
#if LEAD_PA16
  const unsigned int e = __ldg(static_cast<const unsigned short*>(table) + j * V + v);
  p.addr = e & 0x1FFFu;
  p.rank = (e >> 13) & 3u;
  p.first = (e >> 15) != 0;
#else
  const unsigned int e = __ldg(static_cast<const unsigned int*>(table) + j * V + v);
  p.addr = e & 0xFFFFu;
  p.rank = (e >> 16) & 0xFFu;
  p.first = (e >> 31) != 0;
#endif
  return p;
}

__device__ __forceinline__ unsigned int ld_cluster_u32(unsigned int addr) {
  unsigned int v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void red_cluster_or(unsigned int addr, unsigned int v) {
  asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

extern "C" __global__ void __cluster_dims__(LEAD_CLUSTER, 1, 1) __launch_bounds__(LEAD_BLOCK, LEAD_MINBLOCKS)
lead_bp_jit_cluster(const lead::BPJitArgs a) {
  constexpr int NL = LEAD_NL, ML = LEAD_ML, TS = LEAD_TS, C = LEAD_CLUSTER;
  extern __shared__ __align__(16) unsigned int smem[];
  const int V = a.order, wm = a.words_m;
  msg_t* Us = reinterpret_cast<msg_t*>(smem);
  msg_t* Ps = Us + NL * TS;
  msg_t* Ls = Ps + NL * TS;
#if LEAD_ALIAS
  // the staged syndromes live in the posterior array and the correction bits in the array whose
  // sums U are dead when the shot stops (see the single-CTA kernel); the three verdict words
  // follow the messages
  unsigned int* syn_s = reinterpret_cast<unsigned int*>(Ps);
  unsigned int* flags = smem + kMsgBytes / 4;    // three words, meaningful in rank 0 only
#else
  unsigned int* syn_s = smem + kMsgBytes / 4;
  unsigned int* cb = syn_s + wm;
  unsigned int* flags = cb + a.words_n;          // three words, meaningful in rank 0 only
#endif

  const unsigned int rank = cluster_rank();
  const int tid = threadIdx.x;
  const int v = (int)rank * TS + tid;            // global vertex of this thread
  const bool lane_ok = tid < TS && v < V;
  const msg_t* ubase[C];          // every rank's first message array, as generic addresses
#pragma unroll
  for (int r = 0; r < C; ++r) ubase[r] = map_rank_generic(Us, r);
  const unsigned int flag0 = map_rank(flags, 0);
  const float lam_ch = a.use_lead ? 0.0f : lead::channel_llr(a.p);
  const int K = (a.use_lead && a.header) ? __ldg(a.header) : 0;   // classes of the local table
  const long long cid = blockIdx.x / C, ncl = gridDim.x / C;

  for (long long g0 = cid; g0 < a.shots; g0 += ncl) {
    for (int i = tid; i < wm; i += blockDim.x) syn_s[i] = __ldg(a.syn + g0 * wm + i);
    if (tid < 3) flags[tid] = 0u;
    RowMag mag[ML];
    unsigned int meta[ML];
#pragma unroll
    for (int r = 0; r < ML; ++r) {
      mag[r].set(0.0f, 0.0f);
      meta[r] = 0u;
    }
    __syncthreads();
    unsigned int sv = 0;
    if (lane_ok) {
      sv = lead::bit_field(syn_s, v * ML, ML);
#pragma unroll 2
      for (int j = 0; j < NL; ++j) {
        float lj;
        if (a.lam) {
          const int q = __ldg(a.views + v * NL + j);
          lj = lead::in_bounds(a.check, q, a.n, 3) ? __ldg(a.lam + g0 * a.n + q) : 0.0f;
        } else if (a.use_lead) {
          const Partner pt = cluster_partner(a.pa, j, v, V);
          const unsigned int addr = pt.addr, pr = pt.rank;
          const unsigned int jp = addr / TS, vp = pr * TS + (addr - jp * TS);
          const bool ok = lead::in_bounds(a.check, addr, NL * TS, 1) && lead::in_bounds(a.check, pr, C, 4) &&
                          lead::in_bounds(a.check, vp, V, 2);
          const unsigned int svp = ok ? lead::bit_field(syn_s, vp * ML, ML) : 0u;
          lj = merged_prior(a, K, sv * NL + j, svp * NL + jp);
        } else {
          lj = lam_ch;
        }
        Ls[j * TS + tid] = enc(lj);
        Us[j * TS + tid] = enc(0.0f);
      }
    }
    cluster_sync();             // zeroed U and cleared flags visible to the whole cluster
    // One cluster barrier per iteration: the first two message arrays trade roles every
    // iteration in every CTA alike (X at offset xo, Y at NL*TS - xo), as in the single-CTA kernel.
    unsigned int fi = 0;        // verdict word of this iteration (three in rotation)
    for (int t = 0;; ++t) {
      const int xo = (t & 1) ? NL * TS : 0;
      msg_t* X = Us + xo;
      msg_t* Y = Us + (NL * TS - xo);
      HardBits hm;
      unsigned int bad = 0;
      if (lane_ok) {
        // partner sums in groups of kPartnerGroup slots: all reads of a group are issued before
        // any of them is used, so their distributed-shared-memory latencies overlap
        constexpr int G = kPartnerGroup;
#pragma unroll
        for (int j0 = 0; j0 < NL; j0 += G) {
          msg_t upr[G];
          unsigned int first = 0;
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int j = j0 + g;
            if (j < NL) {
              const Partner pt = cluster_partner(a.pa, j, v, V);
              const unsigned int addr = pt.addr, pr = pt.rank;
              const msg_t* ub = ubase[0];
#pragma unroll
              for (int r = 1; r < C; ++r) ub = (pr == (unsigned int)r) ? ubase[r] : ub;
              // ordered after the previous cluster barrier (memory clobber)
              upr[g] = (lead::in_bounds(a.check, addr, NL * TS, 1) && lead::in_bounds(a.check, pr, C, 4))
                           ? ub[xo + addr]
                           : enc(0.0f);
              first |= (unsigned int)pt.first << g;
            }
          }
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int j = j0 + g;
            if (j < NL) {
              const msg_t pe = enc(slot_post((first >> g) & 1u, dec(Ls[j * TS + tid]), dec(X[j * TS + tid]),
                                             dec(upr[g])));
              Y[j * TS + tid] = pe;
              hm.push_neg(j, dec(pe));
            }
          }
        }
#pragma unroll
        for (int r = 0; r < ML; ++r) bad |= (hm.row_parity(r) ^ (sv >> r)) & 1u;
        if (bad) red_cluster_or(flag0 + 4u * fi, 1u);
      }
      const unsigned int fn = fi == 2u ? 0u : fi + 1u;
      if (rank == 0 && tid == 0) flags[fn] = 0u;     // last read two barriers ago
      const bool last = t >= a.max_iter;            // uniform
      if (lane_ok && !last) {
        check_update(mag, meta, sv, Y, tid);
        store_u(mag, meta, Y, tid);
      }
      cluster_sync();           // every CTA's U and every verdict bit in place
      const bool conv = ld_cluster_u32(flag0 + 4u * fi) == 0u;
      if (conv || last) {       // uniform across the cluster: every thread read the same flag
#if LEAD_ALIAS
        unsigned int* cbw = reinterpret_cast<unsigned int*>(Y);
#else
        unsigned int* cbw = cb;
#endif
        for (int i = tid; i < a.words_n; i += blockDim.x) cbw[i] = 0u;
        __syncthreads();
        if (lane_ok) {
          for (int j = 0; j < NL; ++j) {
            const Partner pt = cluster_partner(a.pa, j, v, V);
            if (pt.first) {
              const int q = __ldg(a.views + v * NL + j);
              if (!lead::in_bounds(a.check, q, a.n, 3)) continue;
              if (hm.get(j)) atomicOr(cbw + (q >> 5), 1u << (q & 31));
              if (a.llr) {
                // the posterior of iteration t again, from the same stored operands (no CTA
                // writes its X before the barriers below)
                const msg_t* ub = ubase[0];
#pragma unroll
                for (int r = 1; r < C; ++r) ub = (pt.rank == (unsigned int)r) ? ubase[r] : ub;
                const bool ok = lead::in_bounds(a.check, pt.addr, NL * TS, 1) && lead::in_bounds(a.check, pt.rank, C, 4);
                const float up = ok ? dec(ub[xo + pt.addr]) : 0.0f;
                a.llr[g0 * a.n + q] = rnd(slot_post(true, dec(Ls[j * TS + tid]), dec(X[j * TS + tid]), up));
              }
            }
          }
        }
        if (rank == 0 && tid == 0) {
          a.status[g0] = conv ? (unsigned char)1 : (unsigned char)2;
          if (a.iters) a.iters[g0] = t;
        }
        cluster_sync();         // every CTA's correction bits are in its cbw
        if (rank == 0) {
          for (int i = tid; i < a.words_n; i += blockDim.x) {
            unsigned int w = cbw[i];
#pragma unroll
            for (int r = 1; r < C; ++r) w |= ld_cluster_u32(map_rank(cbw + i, r));
            a.corr[g0 * a.words_n + i] = w;
          }
        }
        cluster_sync();         // rank 0 has read every cbw and every CTA its partners' X
        break;
      }
      fi = fn;
    }
  }
}

}  // namespace lead_jit
#endif
