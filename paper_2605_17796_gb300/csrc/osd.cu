// Ordered-statistics decoding (OSD-CS) after min-sum (the paper's global decoder is BP-OSD,
// osd_cs order 3, Sec. IV-A), for the shots whose min-sum did not converge.
//
// One CTA per shot at a time (persistent over the shots), with the shot's row-reduced check
// matrix in a private workspace slot (bit-packed rows, global memory):
//   1. column order: qubits by ascending BP posterior LLR (order-preserving integer key of the
//      binary32 value), ties by qubit index: a bitonic sort in shared memory;
//   2. Gauss-Jordan elimination over GF(2) in that column order, the syndrome carried along,
//      blocked by 64 columns (the reduced rows are unique, so the pivot row choice is free);
//   3. candidates: OSD-0 (e_T = 0), every single non-basis column, every pair among the first
//      `order` non-basis columns; soft weight sum_{e_i = 1} W_i with W_i = rint(2^20 lambda_i)
//      from the global decoder's binary32 prior, exact integer sums, ties to the earlier one;
//   4. the chosen correction replaces the shot's correction row; status gains LEAD_ST_OSD.
#include <cuda_runtime.h>

#include <algorithm>

#include "lead_device.cuh"

namespace lead {
int check_device(const lead_code* code);

namespace {

constexpr int kOsdThreads = 512;
constexpr int kOsdMaxN = 65535;       // column and row indices are stored as uint16
constexpr int kOsdMaxM = 65535;
constexpr size_t kOsdMaxSmem = 227u * 1024u;
constexpr int kOsdMaxOrder = 6;
constexpr unsigned long long kNone = ~0ull;

struct OsdArgs {
  int n, m, m_l, nl, words_m, words_n, w64, order, rank_max;
  int64_t shots;
  const uint32_t* syn;
  const float* prior;         // shots x n, or null: the channel LLR lam_ch for every qubit
  float lam_ch;
  const float* post;          // shots x n BP posterior LLRs
  uint8_t* status;
  uint32_t* corr;
  const uint16_t* views;      // order x nl qubit ids
  unsigned long long* scratch;  // gridDim.x slots of m x w64 words
  unsigned char* garr;          // gridDim.x slots of the arrays kept in global memory (big codes)
  size_t garr_bytes;            // bytes per slot of garr
  unsigned long long* check;    // checked build: bounds-failure record
};

__device__ __forceinline__ unsigned int order_key(float x) {
  const unsigned int u = __float_as_uint(x);
  return (u >> 31) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ int weight_of(float lam) { return __float2int_rn(__fmul_rn(lam, 1048576.0f)); }

// Block-wide reductions over kOsdThreads threads (scratch: kOsdThreads / 32 entries).
__device__ long long block_sum_ll(long long v, long long* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  long long t = 0;
  for (int i = 0; i < kOsdThreads / 32; ++i) t += red[i];
  __syncthreads();
  return t;
}

// minimum of (cost, index) pairs packed so that the smaller cost wins, then the smaller index
__device__ void block_min_pair(long long& cost, int& idx, long long* redc, int* redi) {
  for (int o = 16; o > 0; o >>= 1) {
    const long long oc = __shfl_xor_sync(0xFFFFFFFFu, cost, o);
    const int oi = __shfl_xor_sync(0xFFFFFFFFu, idx, o);
    if (oc < cost || (oc == cost && oi < idx)) {
      cost = oc;
      idx = oi;
    }
  }
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    redc[w] = cost;
    redi[w] = idx;
  }
  __syncthreads();
  cost = redc[0];
  idx = redi[0];
  for (int i = 1; i < kOsdThreads / 32; ++i)
    if (redc[i] < cost || (redc[i] == cost && redi[i] < idx)) {
      cost = redc[i];
      idx = redi[i];
    }
  __syncthreads();
}

// Layout of one CTA's arrays. The elimination state of every row (panel word, pivot mask, used
// flag, carried syndrome bit), the pivot-column bitmaps and the reduction scratch always live in
// shared memory. The sort keys (later the staged pivot rows), the column order and weights and the
// per-pivot arrays live there too when everything fits (`big` false); otherwise (`big` true) they
// move to the CTA's slot of global scratch, which stays in L1/L2.
struct OsdLayout {
  int np;                                  // sort size: the power of two >= n
  bool big;
  size_t keys, ord, pos, wc, piv, rowof, dval;              // shared (small) or global (big) offsets
  size_t synb, ispiv, solq, panel, amask, used, misc;       // shared offsets
  size_t qrows;                            // big layout: the staged pivot rows in shared memory
  bool qsm;                                //   when they fit there (else the sort keys' space)
  size_t smem, gmem;                                        // bytes of each
};

__host__ __device__ inline OsdLayout osd_layout(int n, int m, bool big) {
  OsdLayout L{};
  L.big = big;
  L.np = 1;
  while (L.np < n) L.np <<= 1;
  size_t so = 0, go = 0;
  auto take = [](size_t& o, size_t bytes) {
    const size_t at = o;
    o = (o + bytes + 15) & ~size_t(15);
    return at;
  };
  size_t& mo = big ? go : so;              // where the movable arrays go
  // the sort keys, later the 64 staged pivot rows of a panel (64 x ceil(n/64) words)
  const size_t w64 = (size_t)(n + 63) / 64;
  L.keys = take(mo, sizeof(unsigned long long) * (L.np > (int)(64 * w64) ? L.np : 64 * w64));
  L.ord = take(mo, sizeof(uint16_t) * n);
  L.pos = take(mo, sizeof(uint16_t) * n);
  L.wc = take(mo, sizeof(int) * n);
  L.piv = take(mo, sizeof(uint16_t) * m);          // pivot column of reduced row r
  L.rowof = take(mo, sizeof(uint16_t) * m);        // physical row holding reduced row r
  L.dval = take(mo, sizeof(int) * m);
  L.synb = take(so, m);
  L.ispiv = take(so, sizeof(uint32_t) * ((n + 31) / 32));
  L.solq = take(so, sizeof(uint32_t) * ((n + 31) / 32));
  L.panel = take(so, sizeof(unsigned long long) * m);   // the current panel word of every row
  L.amask = take(so, sizeof(unsigned long long) * m);   // which of the panel's pivot rows each row took
  L.used = take(so, m);                                 // row already serves as a pivot
  L.misc = take(so, sizeof(long long) * 2 * (kOsdThreads / 32) + 64 + 64 * sizeof(int) + 64);
  // big layout: the staged pivot rows get their own shared area when it fits; read by every warp
  // for every row in phase B, they are the kernel's hottest data
  const size_t qbytes = sizeof(unsigned long long) * 64 * w64;
  L.qsm = big && so + qbytes <= kOsdMaxSmem;
  if (L.qsm) L.qrows = take(so, qbytes);
  L.smem = so;
  L.gmem = (go + 255) / 256 * 256;
  return L;
}

// BIG selects where the movable arrays live (see OsdLayout); a template parameter, so that in
// the shared-memory variant the compiler sees shared-memory addresses. WIDE: rows of more than
// 64 words, applied in 64-word chunks.
template <bool BIG, bool WIDE>
__global__ void __launch_bounds__(kOsdThreads, 2) osd_kernel(OsdArgs a, float p_ch,
                                                          __grid_constant__ const SideParams P) {
  extern __shared__ __align__(16) unsigned char sm[];
  const OsdLayout L = osd_layout(a.n, a.m, BIG);
  unsigned char* mv = BIG ? a.garr + (size_t)blockIdx.x * a.garr_bytes : sm;     // movable arrays
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(mv + L.keys);
  uint16_t* ord = reinterpret_cast<uint16_t*>(mv + L.ord);
  uint16_t* pos = reinterpret_cast<uint16_t*>(mv + L.pos);
  int* Wc = reinterpret_cast<int*>(mv + L.wc);
  uint16_t* piv = reinterpret_cast<uint16_t*>(mv + L.piv);
  uint16_t* rowof = reinterpret_cast<uint16_t*>(mv + L.rowof);
  unsigned long long* panel = reinterpret_cast<unsigned long long*>(sm + L.panel);
  unsigned long long* amask = reinterpret_cast<unsigned long long*>(sm + L.amask);
  uint8_t* used = sm + L.used;
  // staged pivot rows: the sort keys' space, or their own shared area (big layout, when it fits)
  unsigned long long* qrows = (BIG && L.qsm) ? reinterpret_cast<unsigned long long*>(sm + L.qrows) : keys;
  int* dval = reinterpret_cast<int*>(mv + L.dval);
  uint8_t* synb = sm + L.synb;
  uint32_t* ispiv = reinterpret_cast<uint32_t*>(sm + L.ispiv);
  uint32_t* solq = reinterpret_cast<uint32_t*>(sm + L.solq);
  long long* redc = reinterpret_cast<long long*>(sm + L.misc);
  int* redi = reinterpret_cast<int*>(redc + kOsdThreads / 32);
  int* sh = redi + kOsdThreads / 32;          // sh[0..2] pivot search slots, sh[3..] first non-basis columns
  int* kphys = sh + 16;                        // physical rows of the panel's pivots
  uint8_t* synq = reinterpret_cast<uint8_t*>(kphys + 64);
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = bd >> 5;
  const int n = a.n, m = a.m, W = a.w64;
  const int nw32 = (n + 31) / 32;
  const float lam_ch = channel_llr(p_ch);

  for (int64_t shot = blockIdx.x; shot < a.shots; shot += gridDim.x) {
    if (a.status[shot] & LEAD_ST_CONVERGED) continue;      // uniform across the CTA
    unsigned long long* mat = a.scratch + (size_t)blockIdx.x * m * W;
    const float* post = a.post + shot * (int64_t)n;
    const float* prior = a.prior ? a.prior + shot * (int64_t)n : nullptr;
    // 1. column order: ascending (posterior key, qubit)
    for (int i = tid; i < L.np; i += bd)
      keys[i] = i < n ? ((unsigned long long)order_key(__ldg(post + i)) << 32) | (unsigned int)i : kNone;
    for (int i = tid; i < nw32; i += bd) {
      ispiv[i] = 0u;
      solq[i] = 0u;
    }
    __syncthreads();
    for (int k = 2; k <= L.np; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < L.np; i += bd) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const unsigned long long x = keys[i], y = keys[ixj];
            if ((x > y) == ((i & k) == 0)) {
              keys[i] = y;
              keys[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
    for (int c = tid; c < n; c += bd) {
      const int q = (int)(keys[c] & 0xFFFFFFFFull);
      ord[c] = (uint16_t)q;
      pos[q] = (uint16_t)c;
      Wc[c] = weight_of(prior ? __ldg(prior + q) : lam_ch);
    }
    for (int idx = tid; idx < m * W; idx += bd) mat[idx] = 0ull;
    __syncthreads();
    // 2. the check matrix with columns in that order; syndrome bits
    for (int i = tid; i < m; i += bd) {
      const int v = i / a.m_l, r = i - v * a.m_l;
      unsigned long long* row = mat + (size_t)i * W;
      for (int k = 0; k < P.supp_len[r]; ++k) {
        const int q = __ldg(a.views + v * a.nl + P.supp[r][k]);
        if (!in_bounds(a.check, q, n, 20)) continue;
        const int c = pos[q];
        row[c >> 6] |= 1ull << (c & 63);
      }
      synb[i] = (uint8_t)((__ldg(a.syn + shot * a.words_m + (i >> 5)) >> (i & 31)) & 1u);
    }
    __syncthreads();
    // 3. Gauss-Jordan elimination in blocks of 64 columns (one word of every row). The reduced
    // rows of the pivots, in pivot order, and the carried syndrome are unique for a given
    // column order, so any pivot row may be chosen. Phase A eliminates the panel word of every
    // row in shared memory and records, per row, which of the panel's pivot rows (as they
    // stood at the panel's start) it took; phase B applies those sums to the full rows.
    for (int i = tid; i < m; i += bd) used[i] = 0;
    if (tid < 3) sh[tid] = 0x7FFFFFFF;
    __syncthreads();
    // One barrier per column. Thread t owns rows t, t + bd, ...: it eliminates them and then
    // searches them for the next column's pivot at once, so the search sees their current panel
    // words. The pivot of the column processed as the g-th goes through slot g % 3; thread 0 frees
    // slot (g - 1) % 3 after barrier g, when every thread has read it, well before column g + 2
    // searches into it.
    int rank = 0, g = 0;
    for (int pn = 0; pn < W && rank < a.rank_max; ++pn) {
      for (int i = tid; i < m; i += bd) {
        panel[i] = mat[(size_t)i * W + pn];
        amask[i] = 0ull;
      }
      const int bmax = n - pn * 64 < 64 ? n - pn * 64 : 64;
      for (int i = tid; i < m; i += bd)          // the panel's first column, own rows
        if (!used[i] && (panel[i] & 1ull)) {
          atomicMin(sh + g % 3, i);
          break;
        }
      int k = 0;
      for (int b = 0; b < bmax && rank + k < a.rank_max; ++b, ++g) {
        const int col = pn * 64 + b;
        __syncthreads();                                   // column b's slot is final
        const int pr = sh[g % 3];
        if (tid == 0) sh[(g + 2) % 3] = 0x7FFFFFFF;        // column b - 1's slot, read by all
        if (pr != 0x7FFFFFFF) {
          const unsigned long long pp = panel[pr], ap = amask[pr] ^ (1ull << k);
          for (int i = tid; i < m; i += bd)
            if (i != pr && ((panel[i] >> b) & 1ull)) {
              panel[i] ^= pp;
              amask[i] ^= ap;
            }
          if (pr % bd == tid) used[pr] = 1;                 // only the owner reads it
          if (tid == 0) {
            kphys[k] = pr;
            piv[rank + k] = (uint16_t)col;
            rowof[rank + k] = (uint16_t)pr;
            ispiv[col >> 5] |= 1u << (col & 31);
          }
          ++k;
        }
        if (b + 1 < bmax && rank + k < a.rank_max)        // the next column, own rows
          for (int i = tid; i < m; i += bd)
            if (!used[i] && ((panel[i] >> (b + 1)) & 1ull)) {
              atomicMin(sh + (g + 1) % 3, i);
              break;
            }
      }
      __syncthreads();                                     // pivots and panel state visible
      if (k > 0) {
        for (int idx = tid; idx < k * W; idx += bd) {
          const int kk = idx / W, w = idx - kk * W;
          qrows[idx] = mat[(size_t)kphys[kk] * W + w];
        }
        for (int kk = tid; kk < k; kk += bd) synq[kk] = synb[kphys[kk]];
        __syncthreads();
        // warp per row, the row's mask bits walked once per 64-word chunk (warp-uniform), lanes
        // on words w0 + lane and w0 + lane + 32; the row's words are loaded first so the loads are
        // in flight during the walk
        if (!WIDE) {
          const bool has0 = lane < W, has1 = lane + 32 < W;
          for (int i = warp; i < m; i += nwarps) {
            const unsigned long long am = amask[i];
            if (!am) continue;
            unsigned long long* row = mat + (size_t)i * W;
            const unsigned long long r0 = has0 ? row[lane] : 0ull;
            const unsigned long long r1 = has1 ? row[lane + 32] : 0ull;
            unsigned long long acc0 = 0ull, acc1 = 0ull;
            unsigned int sacc = 0;
            for (unsigned long long r = am; r; r &= r - 1) {
              const int kk = __ffsll((long long)r) - 1;
              const unsigned long long* q = qrows + kk * W;
              if (has0) acc0 ^= q[lane];
              if (has1) acc1 ^= q[lane + 32];
              sacc ^= synq[kk];
            }
            if (has0) row[lane] = r0 ^ acc0;
            if (has1) row[lane + 32] = r1 ^ acc1;
            if (lane == 0) synb[i] ^= (uint8_t)sacc;
          }
        } else for (int i = warp; i < m; i += nwarps) {
          const unsigned long long am = amask[i];
          if (!am) continue;
          unsigned long long* row = mat + (size_t)i * W;
          for (int w0 = 0; w0 < W; w0 += 64) {
            const bool has0 = w0 + lane < W, has1 = w0 + lane + 32 < W;
            const unsigned long long r0 = has0 ? row[w0 + lane] : 0ull;
            const unsigned long long r1 = has1 ? row[w0 + lane + 32] : 0ull;
            unsigned long long acc0 = 0ull, acc1 = 0ull;
            unsigned int sacc = 0;
            for (unsigned long long r = am; r; r &= r - 1) {
              const int kk = __ffsll((long long)r) - 1;
              const unsigned long long* q = qrows + (size_t)kk * W + w0;
              if (has0) acc0 ^= q[lane];
              if (has1) acc1 ^= q[lane + 32];
              sacc ^= synq[kk];
            }
            if (has0) row[w0 + lane] = r0 ^ acc0;
            if (has1) row[w0 + lane + 32] = r1 ^ acc1;
            if (w0 == 0 && lane == 0) synb[i] ^= (uint8_t)sacc;
          }
        }
        __syncthreads();
      }
      rank += k;
    }
    __syncthreads();
    // 4. candidate costs
    long long part = 0;
    for (int i = tid; i < rank; i += bd) {
      const int wp = Wc[piv[i]];
      const uint8_t si = synb[rowof[i]];
      dval[i] = si ? -wp : wp;
      part += si ? wp : 0;
    }
    const long long cost0 = block_sum_ll(part, redc);       // (contains the syncs dval needs)
    long long bc = 0x7FFFFFFFFFFFFFFFll;
    int bi = 0x7FFFFFFF;
    for (int c = tid; c < n; c += bd) {
      if ((ispiv[c >> 5] >> (c & 31)) & 1u) continue;
      long long acc = Wc[c];
      const int wc = c >> 6;
      const unsigned long long bit = 1ull << (c & 63);
      for (int i0 = 0; i0 < rank; i0 += 8) {           // eight independent loads in flight
        unsigned long long wv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) wv[u] = i0 + u < rank ? mat[(size_t)rowof[i0 + u] * W + wc] : 0ull;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (wv[u] & bit) acc += dval[i0 + u];
      }
      const long long cost = cost0 + acc;
      if (cost < bc || (cost == bc && c < bi)) {
        bc = cost;
        bi = c;
      }
    }
    block_min_pair(bc, bi, redc, redi);
    if (tid == 0) {
      int cnt = 0;
      for (int c = 0; c < n && cnt < a.order; ++c)
        if (!((ispiv[c >> 5] >> (c & 31)) & 1u)) sh[3 + cnt++] = c;
      sh[3 + kOsdMaxOrder] = cnt;
    }
    __syncthreads();
    long long wcost = cost0;
    int kind = 0, ca = -1, cb = -1;
    if (bi != 0x7FFFFFFF && bc < wcost) {
      wcost = bc;
      kind = 1;
      ca = bi;
    }
    const int nt = sh[3 + kOsdMaxOrder];
    for (int pa = 0; pa < nt; ++pa)
      for (int pb = pa + 1; pb < nt; ++pb) {
        const int x = sh[3 + pa], y = sh[3 + pb];
        long long ps = 0;
        for (int i = tid; i < rank; i += bd) {
          const unsigned long long* row = mat + (size_t)rowof[i] * W;
          if ((((row[x >> 6] >> (x & 63)) ^ (row[y >> 6] >> (y & 63))) & 1ull) != 0) ps += dval[i];
        }
        const long long cost = cost0 + Wc[x] + Wc[y] + block_sum_ll(ps, redc);
        if (cost < wcost) {
          wcost = cost;
          kind = 2;
          ca = x;
          cb = y;
        }
      }
    // 5. the chosen correction, in qubit order
    for (int i = tid; i < rank; i += bd) {
      const unsigned long long* row = mat + (size_t)rowof[i] * W;
      unsigned int v = synb[rowof[i]];
      if (kind >= 1) v ^= (unsigned int)((row[ca >> 6] >> (ca & 63)) & 1ull);
      if (kind == 2) v ^= (unsigned int)((row[cb >> 6] >> (cb & 63)) & 1ull);
      if (v) {
        const int q = ord[piv[i]];
        atomicOr(solq + (q >> 5), 1u << (q & 31));
      }
    }
    if (tid == 0) {
      if (kind >= 1) atomicOr(solq + (ord[ca] >> 5), 1u << (ord[ca] & 31));
      if (kind == 2) atomicOr(solq + (ord[cb] >> 5), 1u << (ord[cb] & 31));
    }
    __syncthreads();
    for (int w = tid; w < a.words_n; w += bd) a.corr[shot * a.words_n + w] = w < nw32 ? solq[w] : 0u;
    if (tid == 0) a.status[shot] = (uint8_t)(a.status[shot] | LEAD_ST_OSD);
    __syncthreads();
  }
}

size_t osd_matrix_bytes(const lead_code* code, int side) {
  const size_t w64 = ((size_t)code->n + 63) / 64;
  return ((size_t)code->side[side].m * w64 * 8 + 255) / 256 * 256;
}

// The layout a side uses: everything in shared memory when it fits, else the movable arrays in
// global scratch.
OsdLayout osd_side_layout(const lead_code* code, int side) {
  const OsdLayout small = osd_layout(code->n, code->side[side].m, false);
  return small.smem <= kOsdMaxSmem ? small : osd_layout(code->n, code->side[side].m, true);
}

// Workspace of one CTA slot: its matrix, then (big codes) its global arrays.
size_t osd_slot_bytes(const lead_code* code, int side) {
  const OsdLayout L = osd_side_layout(code, side);
  return osd_matrix_bytes(code, side) + (L.big ? L.gmem : 0);
}

int osd_slots(const lead_code* code, int64_t shots) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(shots, 2 * (int64_t)sm_count(code->device)));
}

}  // namespace
}  // namespace lead

extern "C" {

size_t lead_osd_workspace_bytes(const lead_code* code, const lead_decode_opts* opts, int64_t shots) {
  if (!code || !opts || opts->side < 0 || opts->side > 1 || shots < 0 || code->device < 0) return 0;
  return (size_t)lead::osd_slots(code, shots) * lead::osd_slot_bytes(code, opts->side);
}

int lead_osd(const lead_code* code, const lead_decode_opts* opts, int32_t order, const uint32_t* syn, int64_t shots,
             const float* prior, const float* post, uint8_t* status, uint32_t* corr, void* workspace,
             size_t ws_bytes, void* stream) {
  using namespace lead;
  int rc = check_device(code);
  if (rc != LEAD_OK) return rc;
  if (!opts || opts->side < 0 || opts->side > 1 || order < 0 || order > kOsdMaxOrder || shots < 0)
    return LEAD_EINVAL;
  const HostSide& hs = code->side[opts->side];
  if (code->n > kOsdMaxN || hs.m > kOsdMaxM) return LEAD_EINVAL;     // uint16 column / row ids
  if (!prior && !(opts->p > 0.0 && opts->p < 0.5)) return LEAD_EINVAL;
  if (shots == 0) return LEAD_OK;
  if (!syn || !post || !status || !corr || !workspace || ((uintptr_t)workspace & 15)) return LEAD_EINVAL;
  const size_t slot = osd_slot_bytes(code, opts->side);
  const int slots = (int)std::min<int64_t>(osd_slots(code, shots), (int64_t)(ws_bytes / slot));
  if (slots < 1) return LEAD_EINVAL;
  const OsdLayout L = osd_side_layout(code, opts->side);
  if (L.smem > kOsdMaxSmem) return LEAD_EINVAL;
  const bool wide = (code->n + 63) / 64 > 64;
  auto* kern = L.big ? osd_kernel<true, true> : (wide ? osd_kernel<false, true> : osd_kernel<false, false>);
  if (L.smem > 48u * 1024u)
    LEAD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
  OsdArgs a{};
  a.n = code->n;
  a.m = hs.m;
  a.m_l = hs.m_l;
  a.nl = code->nl;
  a.words_m = hs.params.words_m;
  a.words_n = code->words_n;
  a.w64 = (code->n + 63) / 64;
  a.order = order;
  a.rank_max = hs.rank;
  a.shots = shots;
  a.syn = syn;
  a.prior = prior;
  a.post = post;
  a.status = status;
  a.corr = corr;
  a.views = code->dside[opts->side].views;
  // slots matrices first, then the slots' global arrays (big codes)
  const size_t mat_bytes = osd_matrix_bytes(code, opts->side);
  a.scratch = static_cast<unsigned long long*>(workspace);
  a.garr_bytes = L.big ? L.gmem : 0;
  a.garr = static_cast<unsigned char*>(workspace) + (size_t)slots * mat_bytes;
  a.check = code->d_check;
  kern<<<slots, kOsdThreads, L.smem, (cudaStream_t)stream>>>(a, (float)(opts->p > 0.0 ? opts->p : 0.25), hs.params);
  LEAD_CUDA_TRY(cudaGetLastError());
  return check_result(code, stream);
}

}  // extern "C"
