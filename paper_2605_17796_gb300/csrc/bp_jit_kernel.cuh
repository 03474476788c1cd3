// Global min-sum decoder (Phase 3 of Algorithm 1, with Phases 1-2 fused into its prologue),
// specialised at run time (NVRTC) to one code side. The generated prelude defines
//   LEAD_NL (Delta^2), LEAD_ML (local rows m_l), LEAD_TS (threads with work = shots per CTA *
//   |G|), LEAD_BLOCK (block size), LEAD_MINBLOCKS (CTAs per SM), LEAD_KMAX, and the
//   constant tables lead_jit::kLen[ML] (row weights), kSupp[ML][KMAX] (local indices of every
//   local row, increasing) and kRowMask[ML] (the same rows as 64-bit masks),
// so every loop over a check's support below has compile-time trip counts and offsets.
//
// Mapping: one CTA handles `spb` shots; thread t = shot sl * |G| + vertex v. Shared memory is
// slot-major with row stride LEAD_TS: word j * TS + t belongs to local index j of thread t.
//   U[j][t]    sum of the messages of the vertex's local rows into its slot j,
//   post[j][t] posterior LLR of the slot,  lam[j][t] prior LLR of the slot.
// The global table pa[j][t] holds the shared-memory address of the partner slot (the qubit's
// other view) with bit 15 set when this view belongs to the smaller vertex. Each thread keeps
// the compressed state of its ML local checks in registers: (min1, min2, meta), meta bits 0..25
// = signs of the v2c messages by support position, 26..30 = position of the first minimum,
// 31 = parity s_c + sum of signs. The message to position k is (-1)^(parity + sign_k) times
// (k == argmin ? min2 : min1), exactly the minimum over the other positions.
//
// Order of operations (identical to the oracle's binary32 decision track):
//   post_i = (lambda_i + U_v0) + U_v1 (v0 < v1 the qubit's two views), U_v accumulated from 0 in
//   increasing local row order; v2c = post - c2v_old; hard decision e_i = [post_i < 0];
//   iteration t tests H e = s first and stops at the first success (t = 0 tests the prior).

#if LEAD_CLUSTER == 1
namespace lead_jit {

extern "C" __global__ void __launch_bounds__(LEAD_BLOCK, LEAD_MINBLOCKS)
lead_bp_jit(const lead::BPJitArgs a) {
  constexpr int NL = LEAD_NL, ML = LEAD_ML, TS = LEAD_TS;
  extern __shared__ __align__(16) unsigned int smem[];
  const int V = a.order, spb = a.spb, wm = a.words_m;
  float* Us = reinterpret_cast<float*>(smem);
  float* Ps = Us + NL * TS;
  float* Ls = Ps + NL * TS;
  unsigned int* syn_s = reinterpret_cast<unsigned int*>(Ls + NL * TS);
  unsigned int* cb = syn_s + spb * wm;
  int* flags = reinterpret_cast<int*>(cb + spb * a.words_n);
  const unsigned short* __restrict__ PA = a.pa;

  const int tid = threadIdx.x;
  const int sl = tid / V, v = tid - sl * V;
  const bool lane_ok = tid < TS;
  const float lam_ch = a.use_lead ? 0.0f : lead::channel_llr(a.p, a.llr_t0, a.llr_t1);

  for (long long g0 = (long long)blockIdx.x * spb; g0 < a.shots; g0 += (long long)gridDim.x * spb) {
    const int nsh = (int)((a.shots - g0) < spb ? (a.shots - g0) : spb);
    for (int i = tid; i < nsh * wm; i += blockDim.x) syn_s[i] = __ldg(a.syn + g0 * wm + i);
    for (int i = tid; i < spb * a.words_n; i += blockDim.x) cb[i] = 0u;
    if (tid < 2 * spb) flags[tid] = 0;
    __syncthreads();
    const bool act = lane_ok && sl < nsh;
    float m1[ML], m2[ML];
    unsigned int meta[ML];
#pragma unroll
    for (int r = 0; r < ML; ++r) {
      m1[r] = 0.0f;
      m2[r] = 0.0f;
      meta[r] = 0u;
    }
    unsigned int sv = 0;
    if (act) {
      const unsigned int* srow = syn_s + sl * wm;
      sv = lead::bit_field(srow, v * ML, ML);
#pragma unroll 2
      for (int j = 0; j < NL; ++j) {
        if (a.lam) {
          Ls[j * TS + tid] = __ldg(a.lam + (g0 + sl) * a.n + __ldg(a.views + v * NL + j));
        } else if (a.use_lead) {
          const unsigned int addr = __ldg(PA + j * TS + tid) & 0x7FFFu;
          const unsigned int jp = addr / TS, vp = addr - jp * TS - sl * V;
          const unsigned int svp = lead::bit_field(srow, vp * ML, ML);
          Ls[j * TS + tid] = lead::merged_llr(__ldg(a.table + sv * NL + j), __ldg(a.table + svp * NL + jp),
                                              a.alpha, a.llr_t0, a.llr_t1);
        } else {
          Ls[j * TS + tid] = lam_ch;
        }
        Us[j * TS + tid] = 0.0f;
      }
    }
    __syncthreads();
    bool mydone = !act;
    for (int t = 0;; ++t) {
      unsigned long long hm = 0;
      unsigned int bad = 0;
      if (!mydone) {
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const unsigned int pa = __ldg(PA + j * TS + tid);
          const float up = Us[pa & 0x7FFFu];
          const float uo = Us[j * TS + tid];
          const float lj = Ls[j * TS + tid];
          const float pj = (pa >> 15) ? __fadd_rn(__fadd_rn(lj, uo), up) : __fadd_rn(__fadd_rn(lj, up), uo);
          Ps[j * TS + tid] = pj;
          hm |= (unsigned long long)(pj < 0.0f) << j;
        }
#pragma unroll
        for (int r = 0; r < ML; ++r) bad |= (unsigned int)(__popcll(hm & kRowMask[r]) ^ (sv >> r)) & 1u;
      }
      bool conv;
      if (LEAD_SPB == 1) {
        // one shot per CTA: the block-wide OR of the local check failures is the shot's verdict
        conv = !__syncthreads_or(bad);
      } else {
        if (bad) atomicOr(flags + (t & 1) * spb + sl, 1);
        if (tid < spb) flags[((t + 1) & 1) * spb + tid] = 0;
        __syncthreads();
        conv = flags[(t & 1) * spb + sl] == 0;
      }
      if (!mydone && (conv || t >= a.max_iter)) {
        const long long shot = g0 + sl;
        for (int j = 0; j < NL; ++j) {
          if (__ldg(PA + j * TS + tid) >> 15) {
            const int q = __ldg(a.views + v * NL + j);
            if ((hm >> j) & 1) atomicOr(cb + sl * a.words_n + (q >> 5), 1u << (q & 31));
            if (a.llr) a.llr[shot * a.n + q] = Ps[j * TS + tid];
          }
        }
        if (v == 0) {
          a.status[shot] = conv ? (unsigned char)1 : (unsigned char)2;
          if (a.iters) a.iters[shot] = t;
        }
        mydone = true;
      }
      if (LEAD_SPB == 1) {
        if (conv || t >= a.max_iter) break;       // uniform across the CTA
      } else {
        if (!__syncthreads_or(!mydone)) break;
      }
      if (!mydone) {
#pragma unroll
        for (int r = 0; r < ML; ++r) {
          const float m1o = m1[r], m2o = m2[r];
          const unsigned int mo = meta[r];
          const int amo = (int)((mo >> 26) & 31u);
          const unsigned int flip = mo ^ (0u - (mo >> 31));   // bit k: sign of the old message to k
          float n1 = __int_as_float(0x7F800000), n2 = __int_as_float(0x7F800000);
          int am = 0;
          unsigned int sg = 0;
#pragma unroll
          for (int k = 0; k < LEAD_KMAX; ++k) {
            if (k >= kLen[r]) break;      // constant after unrolling
            const float mago = (k == amo) ? m2o : m1o;
            const float co = __uint_as_float(__float_as_uint(mago) ^ ((flip >> k) << 31));
            const float v2c = __fsub_rn(Ps[kSupp[r][k] * TS + tid], co);
            const float m = fabsf(v2c);
            // v2c is never -0 (every sum starts from +0 terms): its sign bit equals v2c < 0
            sg |= (__float_as_uint(v2c) >> 31) << k;
            const bool lt = m < n1;
            n2 = lt ? n1 : fminf(n2, m);
            n1 = lt ? m : n1;
            am = lt ? k : am;
          }
          const unsigned int par = ((unsigned int)__popc(sg) ^ (sv >> r)) & 1u;
          m1[r] = n1;
          m2[r] = n2;
          meta[r] = sg | ((unsigned int)am << 26) | (par << 31);
          const unsigned int nflip = sg ^ (0u - par);    // bit k: sign of the new message to k
#pragma unroll
          for (int k = 0; k < LEAD_KMAX; ++k) {
            if (k >= kLen[r]) break;      // constant after unrolling
            const float mag = (k == am) ? n2 : n1;
            const float c = __uint_as_float(__float_as_uint(mag) ^ ((nflip >> k) << 31));
            float* u = Us + kSupp[r][k] * TS + tid;
            // the first local row touching a slot stores, later rows add (0 + c == c exactly)
            *u = kFirst[r][k] ? c : __fadd_rn(*u, c);
          }
        }
      }
      __syncthreads();
    }
    __syncthreads();     // every thread's correction bits are in cb before the copy-out
    for (int i = tid; i < nsh * a.words_n; i += blockDim.x) a.corr[g0 * a.words_n + i] = cb[i];
    __syncthreads();
  }
}

}  // namespace lead_jit
#endif

#if LEAD_CLUSTER > 1
// ---------------------------------------------------------------------------------------------
// The same decoder for codes whose per-shot state exceeds one CTA's shared memory: a cluster of
// LEAD_CLUSTER CTAs handles one shot, CTA rank r owning vertices r*TS .. r*TS + TS - 1 (TS =
// LEAD_TS). A partner slot owned by another CTA is read from that CTA's shared memory through
// the cluster's distributed shared memory (mapa + ld.shared::cluster). The iteration's two
// synchronisation points are cluster barriers; the shot's verdict is one flag word in rank 0,
// OR-ed by every thread with a violated local check and read back by all threads after the
// barrier, so every CTA of the cluster takes the same branch at every step.
// The partner table pa32[j][v] (per global vertex v) holds: bits 0..15 the partner slot's word
// address inside its owner CTA, bits 16..23 the owner's rank, bit 31 set when this view belongs
// to the smaller vertex.
// ---------------------------------------------------------------------------------------------
namespace lead_jit {

__device__ __forceinline__ unsigned int cluster_rank() {
  unsigned int r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned int map_rank(const void* p, unsigned int rank) {
  const unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
  unsigned int out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(a), "r"(rank));
  return out;
}

__device__ __forceinline__ float ld_cluster_f32(unsigned int addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int ld_cluster_u32(unsigned int addr) {
  unsigned int v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void red_cluster_or(unsigned int addr, unsigned int v) {
  asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

extern "C" __global__ void __cluster_dims__(LEAD_CLUSTER, 1, 1) __launch_bounds__(LEAD_BLOCK, LEAD_MINBLOCKS)
lead_bp_jit_cluster(const lead::BPJitArgs a) {
  constexpr int NL = LEAD_NL, ML = LEAD_ML, TS = LEAD_TS, C = LEAD_CLUSTER;
  extern __shared__ __align__(16) unsigned int smem[];
  const int V = a.order, wm = a.words_m;
  float* Us = reinterpret_cast<float*>(smem);
  float* Ps = Us + NL * TS;
  float* Ls = Ps + NL * TS;
  unsigned int* syn_s = reinterpret_cast<unsigned int*>(Ls + NL * TS);
  unsigned int* cb = syn_s + wm;
  unsigned int* flags = cb + a.words_n;          // two words, meaningful in rank 0 only
  const unsigned int* __restrict__ PA = reinterpret_cast<const unsigned int*>(a.pa);

  const unsigned int rank = cluster_rank();
  const int tid = threadIdx.x;
  const int v = (int)rank * TS + tid;            // global vertex of this thread
  const bool lane_ok = tid < TS && v < V;
  unsigned int ubase[C];
#pragma unroll
  for (int r = 0; r < C; ++r) ubase[r] = map_rank(Us, r);
  const unsigned int flag0 = map_rank(flags, 0);
  const float lam_ch = a.use_lead ? 0.0f : lead::channel_llr(a.p, a.llr_t0, a.llr_t1);
  const long long cid = blockIdx.x / C, ncl = gridDim.x / C;

  for (long long g0 = cid; g0 < a.shots; g0 += ncl) {
    for (int i = tid; i < wm; i += blockDim.x) syn_s[i] = __ldg(a.syn + g0 * wm + i);
    for (int i = tid; i < a.words_n; i += blockDim.x) cb[i] = 0u;
    if (tid < 2) flags[tid] = 0u;
    float m1[ML], m2[ML];
    unsigned int meta[ML];
#pragma unroll
    for (int r = 0; r < ML; ++r) {
      m1[r] = 0.0f;
      m2[r] = 0.0f;
      meta[r] = 0u;
    }
    __syncthreads();
    unsigned int sv = 0;
    if (lane_ok) {
      sv = lead::bit_field(syn_s, v * ML, ML);
#pragma unroll 2
      for (int j = 0; j < NL; ++j) {
        if (a.lam) {
          Ls[j * TS + tid] = __ldg(a.lam + g0 * a.n + __ldg(a.views + v * NL + j));
        } else if (a.use_lead) {
          const unsigned int pa = __ldg(PA + j * V + v);
          const unsigned int addr = pa & 0xFFFFu, pr = (pa >> 16) & 0xFFu;
          const unsigned int jp = addr / TS, vp = pr * TS + (addr - jp * TS);
          const unsigned int svp = lead::bit_field(syn_s, vp * ML, ML);
          Ls[j * TS + tid] = lead::merged_llr(__ldg(a.table + sv * NL + j), __ldg(a.table + svp * NL + jp),
                                              a.alpha, a.llr_t0, a.llr_t1);
        } else {
          Ls[j * TS + tid] = lam_ch;
        }
        Us[j * TS + tid] = 0.0f;
      }
    }
    cluster_sync();             // zeroed U and cleared flags visible to the whole cluster
    for (int t = 0;; ++t) {
      unsigned long long hm = 0;
      unsigned int bad = 0;
      if (lane_ok) {
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const unsigned int pa = __ldg(PA + j * V + v);
          const unsigned int addr = pa & 0xFFFFu, pr = (pa >> 16) & 0xFFu;
          unsigned int ub = ubase[0];
#pragma unroll
          for (int r = 1; r < C; ++r) ub = (pr == (unsigned int)r) ? ubase[r] : ub;
          const float up = (pr == rank) ? Us[addr] : ld_cluster_f32(ub + 4u * addr);
          const float uo = Us[j * TS + tid];
          const float lj = Ls[j * TS + tid];
          const float pj = (pa >> 31) ? __fadd_rn(__fadd_rn(lj, uo), up) : __fadd_rn(__fadd_rn(lj, up), uo);
          Ps[j * TS + tid] = pj;
          hm |= (unsigned long long)(pj < 0.0f) << j;
        }
#pragma unroll
        for (int r = 0; r < ML; ++r) bad |= (unsigned int)(__popcll(hm & kRowMask[r]) ^ (sv >> r)) & 1u;
        if (bad) red_cluster_or(flag0 + 4u * (t & 1), 1u);
      }
      if (rank == 0 && tid == 0) flags[(t + 1) & 1] = 0u;
      cluster_sync();
      const bool conv = ld_cluster_u32(flag0 + 4u * (t & 1)) == 0u;
      if (conv || t >= a.max_iter) {
        if (lane_ok) {
          for (int j = 0; j < NL; ++j) {
            if (__ldg(PA + j * V + v) >> 31) {
              const int q = __ldg(a.views + v * NL + j);
              if ((hm >> j) & 1) atomicOr(cb + (q >> 5), 1u << (q & 31));
              if (a.llr) a.llr[g0 * a.n + q] = Ps[j * TS + tid];
            }
          }
        }
        if (rank == 0 && tid == 0) {
          a.status[g0] = conv ? (unsigned char)1 : (unsigned char)2;
          if (a.iters) a.iters[g0] = t;
        }
        break;                  // uniform across the cluster: every thread read the same flag
      }
      if (lane_ok) {
#pragma unroll
        for (int r = 0; r < ML; ++r) {
          const float m1o = m1[r], m2o = m2[r];
          const unsigned int mo = meta[r];
          const int amo = (int)((mo >> 26) & 31u);
          const unsigned int flip = mo ^ (0u - (mo >> 31));
          float n1 = __int_as_float(0x7F800000), n2 = __int_as_float(0x7F800000);
          int am = 0;
          unsigned int sg = 0;
#pragma unroll
          for (int k = 0; k < LEAD_KMAX; ++k) {
            if (k >= kLen[r]) break;
            const float mago = (k == amo) ? m2o : m1o;
            const float co = __uint_as_float(__float_as_uint(mago) ^ ((flip >> k) << 31));
            const float v2c = __fsub_rn(Ps[kSupp[r][k] * TS + tid], co);
            const float m = fabsf(v2c);
            sg |= (__float_as_uint(v2c) >> 31) << k;
            const bool lt = m < n1;
            n2 = lt ? n1 : fminf(n2, m);
            n1 = lt ? m : n1;
            am = lt ? k : am;
          }
          const unsigned int par = ((unsigned int)__popc(sg) ^ (sv >> r)) & 1u;
          m1[r] = n1;
          m2[r] = n2;
          meta[r] = sg | ((unsigned int)am << 26) | (par << 31);
          const unsigned int nflip = sg ^ (0u - par);
#pragma unroll
          for (int k = 0; k < LEAD_KMAX; ++k) {
            if (k >= kLen[r]) break;
            const float mag = (k == am) ? n2 : n1;
            const float c = __uint_as_float(__float_as_uint(mag) ^ ((nflip >> k) << 31));
            float* u = Us + kSupp[r][k] * TS + tid;
            *u = kFirst[r][k] ? c : __fadd_rn(*u, c);
          }
        }
      }
      cluster_sync();           // every CTA's U complete before the next gather
    }
    cluster_sync();             // every CTA's correction bits are in its cb
    if (rank == 0) {
      for (int i = tid; i < a.words_n; i += blockDim.x) {
        unsigned int w = cb[i];
#pragma unroll
        for (int r = 1; r < C; ++r) w |= ld_cluster_u32(map_rank(cb + i, r));
        a.corr[g0 * a.words_n + i] = w;
      }
    }
    cluster_sync();             // rank 0 has read every cb before the next shot clears them
  }
}

}  // namespace lead_jit
#endif
