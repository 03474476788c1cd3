// Phases 1-2 (local estimation + regularised merge) and Phase 3 (global min-sum with a
// bit-packed syndrome check per iteration) of Algorithm 1.
#include <cuda_runtime.h>

#include <algorithm>

#include "lead_device.cuh"

namespace lead {
int check_device(const lead_code* code);
int launch_table(const lead_code* code, int side, double p, float* table, cudaStream_t stream);

namespace {

constexpr int kLocalThreads = 256;
constexpr int kLocalShotBatch = 8;

struct LocalArgs {
  int32_t n, spb_rows;
  float alpha;
  int64_t shots;
  const uint32_t* syn;
  const float* table;
  const uint32_t* qslots;
  float* llr;
};

// Phases 1-2 for every (shot, qubit): the two views' boosted local posteriors are read from the
// per-syndrome table (held in shared memory) and merged into the prior LLR. Each thread keeps
// the view slots of its qubits in registers across all shots of the persistent loop.
template <int NL, int KQ>
__global__ void __launch_bounds__(kLocalThreads)
local_estimate_kernel(LocalArgs a, __grid_constant__ const SideParams P) {
  extern __shared__ __align__(16) uint32_t smem[];
  float* tab = reinterpret_cast<float*>(smem);
  const int tab_n = (1 << P.m_l) * NL;
  uint32_t* syn_s = smem + tab_n;
  for (int i = threadIdx.x; i < tab_n; i += blockDim.x) tab[i] = __ldg(a.table + i);
  uint32_t s0[KQ], s1[KQ];
#pragma unroll
  for (int k = 0; k < KQ; ++k) {
    const int i = threadIdx.x + k * kLocalThreads;
    s0[k] = i < a.n ? __ldg(a.qslots + 2 * i) : 0u;
    s1[k] = i < a.n ? __ldg(a.qslots + 2 * i + 1) : 0u;
  }
  const int wm = P.words_m;
  for (int64_t b0 = (int64_t)blockIdx.x * kLocalShotBatch; b0 < a.shots;
       b0 += (int64_t)gridDim.x * kLocalShotBatch) {
    const int nsh = (int)rows_left(kLocalShotBatch, a.shots - b0);
    __syncthreads();
    for (int i = threadIdx.x; i < nsh * wm; i += blockDim.x) syn_s[i] = __ldg(a.syn + b0 * wm + i);
    __syncthreads();
    for (int sl = 0; sl < nsh; ++sl) {
      const uint32_t* row = syn_s + sl * wm;
      float* out = a.llr + (b0 + sl) * (int64_t)a.n;
#pragma unroll
      for (int k = 0; k < KQ; ++k) {
        const int i = threadIdx.x + k * kLocalThreads;
        if (i < a.n) {
          const uint32_t v0 = s0[k] / NL, j0 = s0[k] - v0 * NL;
          const uint32_t v1 = s1[k] / NL, j1 = s1[k] - v1 * NL;
          const uint32_t q0 = bit_field(row, v0 * P.m_l, P.m_l);
          const uint32_t q1 = bit_field(row, v1 * P.m_l, P.m_l);
          out[i] = merged_llr(tab[q0 * NL + j0], tab[q1 * NL + j1], a.alpha);
        }
      }
    }
  }
}

struct BPArgs {
  int32_t n, words_n, spb, max_iter, use_lead;
  float alpha;
  double p;
  int64_t shots;
  const uint32_t* syn;
  uint32_t* corr;
  uint8_t* status;
  int32_t* iters;
  float* llr;
  const float* table;
  const uint16_t* pa;
  const uint16_t* views;
};

constexpr int kBPMaxThreads = 256;

// Global min-sum for one group of `spb` shots per CTA, one thread per (shot, vertex).
// Shared memory is slot-major with a compile-time row stride TS = spb * |V|: entry (j, t)
// belongs to local index j of thread t (thread t = shot sl * V + vertex v of the group), so the
// threads of a warp touch consecutive words and every own-slot offset is an immediate.
//   U[j][t]    sum of the messages of the vertex's local rows into its slot j,
//   post[j][t] posterior LLR of the slot,  lam[j][t] prior LLR of the slot.
// A per-code global table pa[j][t] (16 bits, read through L1) holds the shared-memory address of
// the partner slot (the other view of the same qubit), with bit 15 set when this view belongs
// to the smaller vertex.
// Each thread keeps the compressed state of its ML local checks in registers:
// (min1, min2, meta) with meta bits 0..25 = signs of the v2c messages by support position,
// 26..30 = position of the first minimum, 31 = parity s_c + sum of signs. The message to
// position k is (-1)^(parity + sign_k) times (k == argmin ? min2 : min1), i.e. exactly the
// minimum over the other positions.
template <int NL, int ML, int TS>
__global__ void __launch_bounds__((TS + 31) / 32 * 32, 3)
bp_kernel(BPArgs a, __grid_constant__ const SideParams P) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int V = P.order, spb = a.spb, wm = P.words_m;
  float* Us = reinterpret_cast<float*>(smem);
  float* Ps = Us + NL * TS;
  float* Ls = Ps + NL * TS;
  uint32_t* syn_s = reinterpret_cast<uint32_t*>(Ls + NL * TS);
  const uint16_t* __restrict__ PA = a.pa;          // [j][t]: partner address | first << 15
  uint32_t* cb = syn_s + spb * wm;
  int* flags = reinterpret_cast<int*>(cb + spb * a.words_n);

  const int tid = threadIdx.x;
  const int sl = tid / V, v = tid - sl * V;
  const bool lane_ok = tid < TS;
  const float lam_ch = a.use_lead ? 0.0f : channel_llr(a.p);

  for (int64_t g0 = (int64_t)blockIdx.x * spb; g0 < a.shots; g0 += (int64_t)gridDim.x * spb) {
    const int nsh = (int)rows_left(spb, a.shots - g0);
    for (int i = tid; i < nsh * wm; i += blockDim.x) syn_s[i] = __ldg(a.syn + g0 * wm + i);
    for (int i = tid; i < spb * a.words_n; i += blockDim.x) cb[i] = 0u;
    if (tid < 2 * spb) flags[tid] = 0;
    __syncthreads();
    const bool act = lane_ok && sl < nsh;
    float m1[ML], m2[ML];
    uint32_t meta[ML];
#pragma unroll
    for (int r = 0; r < ML; ++r) {
      m1[r] = 0.0f;
      m2[r] = 0.0f;
      meta[r] = 0u;
    }
    uint32_t sv = 0;
    if (act) {
      const uint32_t* srow = syn_s + sl * wm;
      sv = bit_field(srow, v * ML, ML);
#pragma unroll 2
      for (int j = 0; j < NL; ++j) {
        if (a.use_lead) {
          const uint32_t addr = __ldg(PA + j * TS + tid) & 0x7FFFu;
          const uint32_t jp = addr / TS, vp = addr - jp * TS - sl * V;
          const uint32_t svp = bit_field(srow, vp * ML, ML);
          Ls[j * TS + tid] = merged_llr(__ldg(a.table + sv * NL + j), __ldg(a.table + svp * NL + jp), a.alpha);
        } else {
          Ls[j * TS + tid] = lam_ch;
        }
        Us[j * TS + tid] = 0.0f;
      }
    }
    __syncthreads();
    bool mydone = !act;
    for (int t = 0;; ++t) {
      uint64_t hm = 0;
      if (!mydone) {
#pragma unroll 4
        for (int j = 0; j < NL; ++j) {
          const uint32_t pa = __ldg(PA + j * TS + tid);
          const float up = Us[pa & 0x7FFFu];
          const float uo = Us[j * TS + tid];
          const float lj = Ls[j * TS + tid];
          const float pj = (pa >> 15) ? __fadd_rn(__fadd_rn(lj, uo), up)
                                      : __fadd_rn(__fadd_rn(lj, up), uo);
          Ps[j * TS + tid] = pj;
          hm |= (uint64_t)(pj < 0.0f) << j;
        }
        uint32_t bad = 0;
#pragma unroll
        for (int r = 0; r < ML; ++r) bad |= (uint32_t)(__popcll(hm & P.rowmask[r]) ^ (sv >> r)) & 1u;
        if (bad) atomicOr(flags + (t & 1) * spb + sl, 1);
      }
      if (tid < spb) flags[((t + 1) & 1) * spb + tid] = 0;
      __syncthreads();
      if (!mydone) {
        const bool conv = flags[(t & 1) * spb + sl] == 0;
        if (conv || t >= a.max_iter) {
          const int64_t shot = g0 + sl;
          for (int j = 0; j < NL; ++j) {
            if (__ldg(PA + j * TS + tid) >> 15) {
              const int q = __ldg(a.views + v * NL + j);
              if ((hm >> j) & 1) atomicOr(cb + sl * a.words_n + (q >> 5), 1u << (q & 31));
              if (a.llr) a.llr[shot * a.n + q] = Ps[j * TS + tid];
            }
          }
          if (v == 0) {
            a.status[shot] = conv ? (uint8_t)LEAD_ST_CONVERGED : (uint8_t)LEAD_ST_MAX_ITER;
            if (a.iters) a.iters[shot] = t;
          }
          mydone = true;
        }
      }
      if (!__syncthreads_or(!mydone)) break;
      if (!mydone) {
#pragma unroll 4
        for (int j = 0; j < NL; ++j) Us[j * TS + tid] = 0.0f;
#pragma unroll
        for (int r = 0; r < ML; ++r) {
          const float m1o = m1[r], m2o = m2[r];
          const uint32_t mo = meta[r];
          const int amo = (int)((mo >> 26) & 31u);
          // bit k of `flip` = sign of the old message to position k (parity + sign_k)
          uint32_t flip = mo ^ (0u - (mo >> 31));
          const int len = P.supp_len[r];
          float n1 = __int_as_float(0x7F800000), n2 = __int_as_float(0x7F800000);
          int am = 0;
          uint32_t sg = 0;
          for (int k = 0; k < len; ++k) {
            const float mago = (k == amo) ? m2o : m1o;
            const float co = __uint_as_float(__float_as_uint(mago) ^ (flip << 31));
            flip >>= 1;
            const float v2c = __fsub_rn(Ps[P.supp[r][k] * TS + tid], co);
            const float m = fabsf(v2c);
            // sign bits collect from the top: after the loop bit (32 - len + k) holds position k.
            // v2c is never -0 (every sum starts from +0 terms), so its sign bit equals v2c < 0.
            sg = (sg >> 1) | (__float_as_uint(v2c) & 0x80000000u);
            const bool lt = m < n1;
            n2 = lt ? n1 : fminf(n2, m);
            n1 = lt ? m : n1;
            am = lt ? k : am;
          }
          sg >>= (32 - len);
          const uint32_t par = ((uint32_t)__popc(sg) ^ (sv >> r)) & 1u;
          m1[r] = n1;
          m2[r] = n2;
          meta[r] = sg | ((uint32_t)am << 26) | (par << 31);
          uint32_t nflip = sg ^ (0u - par);
          for (int k = 0; k < len; ++k) {
            const float mag = (k == am) ? n2 : n1;
            const float c = __uint_as_float(__float_as_uint(mag) ^ (nflip << 31));
            nflip >>= 1;
            float* u = Us + P.supp[r][k] * TS + tid;
            *u = __fadd_rn(*u, c);
          }
        }
      }
      __syncthreads();
    }
    for (int i = tid; i < nsh * a.words_n; i += blockDim.x) a.corr[g0 * a.words_n + i] = cb[i];
    __syncthreads();
  }
}

size_t bp_smem_bytes(const lead_code* code, int side, int spb, int threads) {
  const SideParams& P = code->side[side].params;
  return sizeof(uint32_t) * ((size_t)threads * code->nl * 3 + (size_t)spb * P.words_m +
                             (size_t)spb * code->words_n + 2 * (size_t)spb);
}

}  // namespace

int bp_shots_per_block(const lead_code* code) {
  return std::max(1, 256 / code->order);
}

namespace {

size_t table_bytes(const lead_code* code, int side) {
  const size_t b = (size_t)(1 << code->side[side].m_l) * code->nl * sizeof(float);
  return (b + 255) / 256 * 256;
}

int validate_opts(const lead_code* code, const lead_decode_opts* o) {
  if (!o || o->side < 0 || o->side > 1) return LEAD_EINVAL;
  if (o->max_iter < 0 || o->max_iter > kMaxIter) return LEAD_EINVAL;
  if (!(o->alpha > 0.0f && o->alpha <= 1.0f)) return LEAD_EINVAL;
  if (!(o->p > 0.0 && o->p < 0.5)) return LEAD_EINVAL;
  if (o->precision != LEAD_PREC_FP32) return LEAD_EINVAL;
  if (code->nl != 16 && code->nl != 36) return LEAD_EINVAL;
  return LEAD_OK;
}

template <typename K>
int set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    LEAD_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return LEAD_OK;
}

template <int NL>
int launch_local(const lead_code* code, const lead_decode_opts* o, const uint32_t* syn, int64_t shots,
                 float* llr, const float* table, cudaStream_t stream) {
  const SideParams& P = code->side[o->side].params;
  LocalArgs a{};
  a.n = code->n;
  a.alpha = o->alpha;
  a.shots = shots;
  a.syn = syn;
  a.table = table;
  a.qslots = code->dside[o->side].qslots;
  a.llr = llr;
  const size_t smem = sizeof(uint32_t) * ((size_t)(1 << P.m_l) * NL + (size_t)kLocalShotBatch * P.words_m);
  const int kq = (code->n + kLocalThreads - 1) / kLocalThreads;
  auto pick = [&](auto kern) -> int {
    int rc = set_smem(kern, smem);
    if (rc != LEAD_OK) return rc;
    int per_sm = 0;
    LEAD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLocalThreads, smem));
    per_sm = std::max(per_sm, 1);
    const int64_t batches = (shots + kLocalShotBatch - 1) / kLocalShotBatch;
    const int64_t blocks = std::min<int64_t>(batches, (int64_t)sm_count(code->device) * per_sm);
    kern<<<(unsigned)blocks, kLocalThreads, smem, stream>>>(a, P);
    LEAD_CUDA_TRY(cudaGetLastError());
    return LEAD_OK;
  };
  if (kq <= 2) return pick(local_estimate_kernel<NL, 2>);
  if (kq <= 4) return pick(local_estimate_kernel<NL, 4>);
  if (kq <= 12) return pick(local_estimate_kernel<NL, 12>);
  if (kq <= 48) return pick(local_estimate_kernel<NL, 48>);
  return LEAD_EINVAL;
}

template <int NL, int ML, int TS>
int launch_bp(const lead_code* code, const lead_decode_opts* o, const uint32_t* syn, int64_t shots,
              uint32_t* corr, uint8_t* status, int32_t* iters, float* llr, const float* table,
              cudaStream_t stream) {
  const SideParams& P = code->side[o->side].params;
  BPArgs a{};
  a.n = code->n;
  a.words_n = code->words_n;
  a.spb = bp_shots_per_block(code);
  a.max_iter = o->max_iter;
  a.use_lead = o->use_lead ? 1 : 0;
  a.alpha = o->alpha;
  a.p = o->p;
  a.shots = shots;
  a.syn = syn;
  a.corr = corr;
  a.status = status;
  a.iters = iters;
  a.llr = llr;
  a.table = table;
  a.pa = code->dside[o->side].bp_pa;
  a.views = code->dside[o->side].views;
  if (a.spb * P.order != TS || P.m_l != ML || !a.pa) return LEAD_EINVAL;
  const int threads = (TS + 31) / 32 * 32;
  const size_t smem = bp_smem_bytes(code, o->side, a.spb, TS);
  if (smem > 227 * 1024) return LEAD_EINVAL;
  int rc = set_smem(bp_kernel<NL, ML, TS>, smem);
  if (rc != LEAD_OK) return rc;
  int per_sm = 0;
  LEAD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bp_kernel<NL, ML, TS>, threads, smem));
  if (per_sm < 1) return LEAD_EINVAL;
  const int64_t groups = (shots + a.spb - 1) / a.spb;
  const int64_t blocks = std::min<int64_t>(groups, (int64_t)sm_count(code->device) * per_sm);
  bp_kernel<NL, ML, TS><<<(unsigned)blocks, threads, smem, stream>>>(a, P);
  LEAD_CUDA_TRY(cudaGetLastError());
  return LEAD_OK;
}

}  // namespace
}  // namespace lead

extern "C" {

size_t lead_workspace_bytes(const lead_code* code, const lead_decode_opts* opts, int64_t shots) {
  (void)shots;
  if (!code || !opts || opts->side < 0 || opts->side > 1) return 0;
  return opts->use_lead ? lead::table_bytes(code, opts->side) : 0;
}

int lead_local_estimate(const lead_code* code, const lead_decode_opts* opts, const uint32_t* syn,
                        int64_t shots, float* llr, void* workspace, size_t ws_bytes, void* stream) {
  using namespace lead;
  int rc = check_device(code);
  if (rc != LEAD_OK) return rc;
  rc = validate_opts(code, opts);
  if (rc != LEAD_OK) return rc;
  if (shots < 0) return LEAD_EINVAL;
  if (shots == 0) return LEAD_OK;          // empty batch: nothing to read or write
  if (!syn || !llr || !workspace) return LEAD_EINVAL;
  if (((uintptr_t)workspace & 15) || ws_bytes < table_bytes(code, opts->side)) return LEAD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  float* table = static_cast<float*>(workspace);
  rc = launch_table(code, opts->side, opts->p, table, s);
  if (rc != LEAD_OK) return rc;
  if (code->nl == 16) return launch_local<16>(code, opts, syn, shots, llr, table, s);
  return launch_local<36>(code, opts, syn, shots, llr, table, s);
}

int lead_decode(const lead_code* code, const lead_decode_opts* opts, const uint32_t* syn,
                int64_t shots, uint32_t* corr, uint8_t* status, int32_t* iters, float* llr,
                void* workspace, size_t ws_bytes, void* stream) {
  using namespace lead;
  int rc = check_device(code);
  if (rc != LEAD_OK) return rc;
  rc = validate_opts(code, opts);
  if (rc != LEAD_OK) return rc;
  if (shots < 0) return LEAD_EINVAL;
  if (shots == 0) return LEAD_OK;          // empty batch: nothing to read or write
  if (!syn || !corr || !status) return LEAD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  float* table = nullptr;
  if (opts->use_lead) {
    if (!workspace || ((uintptr_t)workspace & 15) || ws_bytes < table_bytes(code, opts->side))
      return LEAD_EINVAL;
    table = static_cast<float*>(workspace);
    rc = launch_table(code, opts->side, opts->p, table, s);
    if (rc != LEAD_OK) return rc;
  }
  const int ml = code->side[opts->side].m_l;
  const int ts = bp_shots_per_block(code) * code->order;
  if (code->nl == 16 && ml == 4 && ts == 240)      // |G| = 24 (SL(2,3)), 10 shots per CTA
    return launch_bp<16, 4, 240>(code, opts, syn, shots, corr, status, iters, llr, table, s);
  if (code->nl == 36 && ml == 9 && ts == 168)      // |G| = 168 (PSL(2,7)), 1 shot per CTA
    return launch_bp<36, 9, 168>(code, opts, syn, shots, corr, status, iters, llr, table, s);
  return LEAD_EINVAL;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Non-allocating decode. Some callers cannot allocate device memory for the workspace: a
// quantum-error-correction control loop whose decode deadline leaves no room for cudaMalloc
// (which may block and synchronise the device), or a host framework whose pool allocator owns
// every byte of device memory. For them the local posterior table lives in a fixed file-scope
// device array instead of the caller's workspace.
// ---------------------------------------------------------------------------------------------
#include <mutex>

namespace lead {
namespace {

constexpr int kNoAllocMaxDevices = 64;
static_assert(LEAD_NOALLOC_TABLE_BYTES % 256 == 0, "table scratch must be a whole number of 256-byte blocks");

// Shared by every call on a device and kept until the process exits; holds the last call's table.
static __device__ __align__(256) float g_noalloc_table[LEAD_NOALLOC_TABLE_BYTES / sizeof(float)];

std::mutex g_noalloc_mu;
float* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Host-side address of the device array on the current device (set up once per device; the
// array's name in host code is only a stand-in and must never be passed to a kernel).
int noalloc_table(int device, float** out) {
  if (device < 0 || device >= kNoAllocMaxDevices) return LEAD_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_table) != cudaSuccess || !p) return LEAD_ECUDA;
    g_noalloc_addr[device] = static_cast<float*>(p);
  }
  *out = g_noalloc_addr[device];
  return LEAD_OK;
}

}  // namespace
}  // namespace lead

extern "C" int lead_decode_noalloc(const lead_code* code, const lead_decode_opts* opts,
                                   const uint32_t* syn, int64_t shots, uint32_t* corr,
                                   uint8_t* status, int32_t* iters, float* llr, void* stream) {
  using namespace lead;
  int rc = check_device(code);
  if (rc != LEAD_OK) return rc;
  rc = validate_opts(code, opts);
  if (rc != LEAD_OK) return rc;
  if (shots < 0) return LEAD_EINVAL;
  if (opts->use_lead && table_bytes(code, opts->side) > (size_t)LEAD_NOALLOC_TABLE_BYTES) return LEAD_EINVAL;
  float* table = nullptr;
  if (opts->use_lead) {
    rc = noalloc_table(code->device, &table);
    if (rc != LEAD_OK) return rc;
  }
  if (shots == 0) return LEAD_OK;
  if (!syn || !corr || !status) return LEAD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (opts->use_lead) {
    rc = launch_table(code, opts->side, opts->p, table, s);
    if (rc != LEAD_OK) return rc;
  }
  const int ml = code->side[opts->side].m_l;
  const int ts = bp_shots_per_block(code) * code->order;
  if (code->nl == 16 && ml == 4 && ts == 240)
    return launch_bp<16, 4, 240>(code, opts, syn, shots, corr, status, iters, llr, table, s);
  if (code->nl == 36 && ml == 9 && ts == 168)
    return launch_bp<36, 9, 168>(code, opts, syn, shots, corr, status, iters, llr, table, s);
  return LEAD_EINVAL;
}
