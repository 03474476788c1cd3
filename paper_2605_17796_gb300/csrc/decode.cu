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
  const uint32_t* partner;
  const uint16_t* views;
};

// Global min-sum for one group of `spb` shots per CTA, one thread per (shot, vertex).
// Shared memory per shot: U[v][j] (sum of the messages of v's local rows into slot j),
// post[v][j] (posterior LLR of slot j), and the compressed state of every check:
// (min1, min2, meta) with meta bits 0..25 = signs of v2c by support position, 26..30 = position
// of the first minimum, 31 = parity s_c + sum of signs. A message to position k is
// (-1)^(parity + sign_k) * (k == argmin ? min2 : min1), i.e. exactly the min over the others.
constexpr int kBPMaxThreads = 256;

template <int NL>
__global__ void __launch_bounds__(kBPMaxThreads)
bp_kernel(BPArgs a, __grid_constant__ const SideParams P) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int V = P.order, ml = P.m_l, spb = a.spb, wm = P.words_m;
  float* U = reinterpret_cast<float*>(smem);
  float* post_s = U + spb * V * NL;
  uint32_t* S = reinterpret_cast<uint32_t*>(post_s + spb * V * NL);
  uint32_t* syn_s = S + spb * V * ml * 3;
  uint32_t* cb = syn_s + spb * wm;
  int* flags = reinterpret_cast<int*>(cb + spb * a.words_n);

  const int tid = threadIdx.x;
  const int sl = tid / V, v = tid - sl * V;
  const bool lane_ok = sl < spb;
  uint32_t part[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) part[j] = lane_ok ? __ldg(a.partner + v * NL + j) : 0u;
  const float lam_ch = a.use_lead ? 0.0f : channel_llr(a.p);
  const int shot_slots = sl * V * NL;
  const int own = shot_slots + v * NL;
  uint32_t* st_base = S + (size_t)(sl * V + v) * ml * 3;

  for (int64_t g0 = (int64_t)blockIdx.x * spb; g0 < a.shots; g0 += (int64_t)gridDim.x * spb) {
    const int nsh = (int)rows_left(spb, a.shots - g0);
    for (int i = tid; i < nsh * wm; i += blockDim.x) syn_s[i] = __ldg(a.syn + g0 * wm + i);
    for (int i = tid; i < spb * a.words_n; i += blockDim.x) cb[i] = 0u;
    if (tid < 2 * spb) flags[tid] = 0;
    __syncthreads();
    const bool act = lane_ok && sl < nsh;
    float lam[NL];
    uint32_t sv = 0;
    if (act) {
      const uint32_t* srow = syn_s + sl * wm;
      sv = bit_field(srow, v * ml, ml);
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        if (a.use_lead) {
          const uint32_t ps = part[j] & 0x7FFFFFFFu;
          const uint32_t vp = ps / NL, jp = ps - vp * NL;
          const uint32_t svp = bit_field(srow, vp * ml, ml);
          lam[j] = merged_llr(__ldg(a.table + sv * NL + j), __ldg(a.table + svp * NL + jp), a.alpha);
        } else {
          lam[j] = lam_ch;
        }
        U[own + j] = 0.0f;
      }
      for (int i = 0; i < ml * 3; ++i) st_base[i] = 0u;
    } else {
#pragma unroll
      for (int j = 0; j < NL; ++j) lam[j] = 0.0f;
    }
    __syncthreads();
    bool mydone = !act;
    for (int t = 0;; ++t) {
      uint64_t hm = 0;
      if (!mydone) {
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const uint32_t ps = part[j];
          const float up = U[shot_slots + (ps & 0x7FFFFFFFu)];
          const float uo = U[own + j];
          const float pj = (ps >> 31) ? __fadd_rn(__fadd_rn(lam[j], uo), up)
                                      : __fadd_rn(__fadd_rn(lam[j], up), uo);
          post_s[own + j] = pj;
          hm |= (uint64_t)(pj < 0.0f) << j;
        }
        uint32_t bad = 0;
        for (int r = 0; r < ml; ++r) bad |= (uint32_t)(__popcll(hm & P.rowmask[r]) ^ (sv >> r)) & 1u;
        if (bad) atomicOr(flags + (t & 1) * spb + sl, 1);
      }
      if (tid < spb) flags[((t + 1) & 1) * spb + tid] = 0;
      __syncthreads();
      if (!mydone) {
        const bool conv = flags[(t & 1) * spb + sl] == 0;
        if (conv || t >= a.max_iter) {
          const int64_t shot = g0 + sl;
#pragma unroll
          for (int j = 0; j < NL; ++j) {
            if (part[j] >> 31) {
              const int q = __ldg(a.views + v * NL + j);
              if ((hm >> j) & 1) atomicOr(cb + sl * a.words_n + (q >> 5), 1u << (q & 31));
              if (a.llr) a.llr[shot * a.n + q] = post_s[own + j];
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
#pragma unroll
        for (int j = 0; j < NL; ++j) U[own + j] = 0.0f;
        for (int r = 0; r < ml; ++r) {
          uint32_t* st = st_base + r * 3;
          const float m1o = __uint_as_float(st[0]), m2o = __uint_as_float(st[1]);
          const uint32_t mo = st[2];
          const int amo = (int)((mo >> 26) & 31u);
          const uint32_t paro = mo >> 31;
          const int len = P.supp_len[r];
          float m1 = __int_as_float(0x7F800000), m2 = __int_as_float(0x7F800000);
          int am = 0;
          uint32_t sg = 0;
          for (int k = 0; k < len; ++k) {
            const int j = P.supp[r][k];
            const float mago = (k == amo) ? m2o : m1o;
            const float co = ((paro ^ (mo >> k)) & 1u) ? -mago : mago;
            const float v2c = __fsub_rn(post_s[own + j], co);
            const float m = fabsf(v2c);
            sg |= (uint32_t)(v2c < 0.0f) << k;
            if (m < m1) {
              m2 = m1;
              m1 = m;
              am = k;
            } else if (m < m2) {
              m2 = m;
            }
          }
          const uint32_t par = ((uint32_t)__popc(sg) ^ (sv >> r)) & 1u;
          st[0] = __float_as_uint(m1);
          st[1] = __float_as_uint(m2);
          st[2] = sg | ((uint32_t)am << 26) | (par << 31);
          for (int k = 0; k < len; ++k) {
            const int j = P.supp[r][k];
            const float mag = (k == am) ? m2 : m1;
            const float c = ((par ^ (sg >> k)) & 1u) ? -mag : mag;
            U[own + j] = __fadd_rn(U[own + j], c);
          }
        }
      }
      __syncthreads();
    }
    for (int i = tid; i < nsh * a.words_n; i += blockDim.x) a.corr[g0 * a.words_n + i] = cb[i];
    __syncthreads();
  }
}

size_t bp_smem_bytes(const lead_code* code, int side, int spb) {
  const SideParams& P = code->side[side].params;
  return sizeof(uint32_t) * ((size_t)spb * P.order * code->nl * 2 + (size_t)spb * P.order * P.m_l * 3 +
                             (size_t)spb * P.words_m + (size_t)spb * code->words_n + 2 * (size_t)spb);
}

int bp_shots_per_block(const lead_code* code) {
  return std::max(1, 256 / code->order);
}

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

template <int NL>
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
  a.partner = code->dside[o->side].partner;
  a.views = code->dside[o->side].views;
  const size_t smem = bp_smem_bytes(code, o->side, a.spb);
  if (smem > 227 * 1024) return LEAD_EINVAL;
  const int threads = (a.spb * P.order + 31) / 32 * 32;
  if (threads > kBPMaxThreads) return LEAD_EINVAL;
  int rc = set_smem(bp_kernel<NL>, smem);
  if (rc != LEAD_OK) return rc;
  int per_sm = 0;
  LEAD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bp_kernel<NL>, threads, smem));
  if (per_sm < 1) return LEAD_EINVAL;
  const int64_t groups = (shots + a.spb - 1) / a.spb;
  const int64_t blocks = std::min<int64_t>(groups, (int64_t)sm_count(code->device) * per_sm);
  bp_kernel<NL><<<(unsigned)blocks, threads, smem, stream>>>(a, P);
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
  if (code->nl == 16) return launch_bp<16>(code, opts, syn, shots, corr, status, iters, llr, table, s);
  return launch_bp<36>(code, opts, syn, shots, corr, status, iters, llr, table, s);
}

}  // extern "C"
