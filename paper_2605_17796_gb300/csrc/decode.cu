// Phases 1-2 (local estimation + regularised merge) and Phase 3 (global min-sum with a
// bit-packed syndrome check per iteration) of Algorithm 1.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "bp_jit_args.h"
#include "lead_device.cuh"

namespace lead {
int check_device(const lead_code* code);
int launch_table(const lead_code* code, int side, double p, float* table, cudaStream_t stream, int estimator,
                 int32_t* iters);
int launch_local_pair(const lead_code* code, const lead_decode_opts* o, const uint32_t* syn, int64_t shots,
                      void* llr, const float* table, void* extra, cudaStream_t stream);

namespace {

constexpr int kLocalThreads = 512;
constexpr int kLocalShotBatch = 32;

struct LocalArgs {
  int32_t n, order;
  float alpha;
  int64_t shots;
  const uint32_t* syn;
  const float* table;
  const uint32_t* qslots;
  void* llr;                    // float, or the 16-bit pattern of the storage format
};

// Store an LLR in the precision mode's storage format (round to nearest even).
template <int PREC>
__device__ __forceinline__ void store_llr(void* base, int64_t idx, float v) {
  if constexpr (PREC == LEAD_PREC_BF16)
    __stcs(static_cast<unsigned short*>(base) + idx, __bfloat16_as_ushort(__float2bfloat16_rn(v)));
  else if constexpr (PREC == LEAD_PREC_FP16)   // saturating at the largest finite binary16
    __stcs(static_cast<unsigned short*>(base) + idx,
           __half_as_ushort(__float2half_rn(fminf(fmaxf(v, -65504.0f), 65504.0f))));
  else
    __stcs(static_cast<float*>(base) + idx, v);
}

// Phases 1-2 for every (shot, qubit): per batch of shots, the local syndromes s_v of all
// vertices are extracted once into shared memory; then every qubit reads its two views'
// boosted local posteriors from the per-syndrome table (shared memory) and merges them into
// the prior LLR. Each thread keeps its qubits' view coordinates in registers for the whole
// persistent loop; the LLR rows are written with consecutive threads on consecutive qubits.
template <int NL, int KQ, int PREC>
__global__ void __launch_bounds__(kLocalThreads, 2)
local_estimate_kernel(LocalArgs a, __grid_constant__ const SideParams P) {
  extern __shared__ __align__(16) uint32_t smem[];
  float* tab = reinterpret_cast<float*>(smem);
  const int tab_n = (1 << P.m_l) * NL;
  uint16_t* sv_s = reinterpret_cast<uint16_t*>(tab + tab_n);   // [batch shot][vertex]
  for (int i = threadIdx.x; i < tab_n; i += blockDim.x) tab[i] = __ldg(a.table + i);
  uint32_t vv[KQ], jj[KQ];       // (v0 | v1 << 16), (j0 | j1 << 16)
#pragma unroll
  for (int k = 0; k < KQ; ++k) {
    const int i = threadIdx.x + k * kLocalThreads;
    const uint32_t s0 = i < a.n ? __ldg(a.qslots + 2 * i) : 0u;
    const uint32_t s1 = i < a.n ? __ldg(a.qslots + 2 * i + 1) : 0u;
    vv[k] = (s0 / NL) | ((s1 / NL) << 16);
    jj[k] = (s0 % NL) | ((s1 % NL) << 16);
  }
  const int wm = P.words_m, V = a.order, ml = P.m_l;
  for (int64_t b0 = (int64_t)blockIdx.x * kLocalShotBatch; b0 < a.shots;
       b0 += (int64_t)gridDim.x * kLocalShotBatch) {
    const int nsh = rows_left(kLocalShotBatch, a.shots - b0);
    __syncthreads();
    for (int i = threadIdx.x; i < nsh * V; i += blockDim.x) {
      const int sl = i / V, v = i - sl * V;
      sv_s[i] = (uint16_t)bit_field(a.syn + (b0 + sl) * wm, v * ml, ml);
    }
    __syncthreads();
#pragma unroll 4
    for (int sl = 0; sl < nsh; ++sl) {
      const uint16_t* svr = sv_s + sl * V;
      const int64_t row = (b0 + sl) * (int64_t)a.n;
#pragma unroll
      for (int k = 0; k < KQ; ++k) {
        const int i = threadIdx.x + k * kLocalThreads;
        if (i < a.n) {
          const float q0 = tab[svr[vv[k] & 0xFFFFu] * NL + (jj[k] & 0xFFFFu)];
          const float q1 = tab[svr[vv[k] >> 16] * NL + (jj[k] >> 16)];
          store_llr<PREC>(a.llr, row + i, merged_llr(q0, q1, a.alpha));
        }
      }
    }
  }
}

}  // namespace

int bp_shots_per_block(const lead_code* code) {
  return std::max(1, std::min(16, 256 / code->order));     // at most 64 after autotuning (x4)
}

namespace {

// The local posterior table (a multiple of 256 bytes); its class tables follow it.
size_t table_bytes(const lead_code* code, int side) {
  const size_t b = (size_t)(1 << code->side[side].m_l) * code->nl * sizeof(float);
  return (b + 255) / 256 * 256;
}

}  // namespace

size_t table_bytes_of(const lead_code* code, int side) { return table_bytes(code, side); }

// The workspace lead_decode reads: the local posterior table and its class tables.
size_t decode_workspace_bytes(const lead_code* code, int side) {
  return table_bytes(code, side) + local_pair_extra_bytes(code, side);
}

namespace {

int validate_opts(const lead_code* code, const lead_decode_opts* o) {
  if (!o || o->side < 0 || o->side > 1) return LEAD_EINVAL;
  if (o->max_iter < 0 || o->max_iter > kMaxIter) return LEAD_EINVAL;
  if (!(o->alpha > 0.0f && o->alpha <= 1.0f)) return LEAD_EINVAL;
  if (!(o->p > 0.0 && o->p < 0.5)) return LEAD_EINVAL;
  if (o->precision != LEAD_PREC_FP32 && o->precision != LEAD_PREC_BF16 && o->precision != LEAD_PREC_FP16)
    return LEAD_EINVAL;
  if (o->estimator != LEAD_EST_EXACT && o->estimator != LEAD_EST_MINSUM) return LEAD_EINVAL;
  if (code->nl != 16 && code->nl != 36) return LEAD_EINVAL;
  return LEAD_OK;
}

template <typename K>
int set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    LEAD_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return LEAD_OK;
}

template <int NL, int PREC>
int launch_local(const lead_code* code, const lead_decode_opts* o, const uint32_t* syn, int64_t shots,
                 void* llr, const float* table, cudaStream_t stream) {
  const SideParams& P = code->side[o->side].params;
  LocalArgs a{};
  a.n = code->n;
  a.order = code->order;
  a.alpha = o->alpha;
  a.shots = shots;
  a.syn = syn;
  a.table = table;
  a.qslots = code->dside[o->side].qslots;
  a.llr = llr;
  const size_t smem = sizeof(uint32_t) * (size_t)(1 << P.m_l) * NL +
                      sizeof(uint16_t) * (size_t)kLocalShotBatch * code->order;
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
  if (kq <= 1) return pick(local_estimate_kernel<NL, 1, PREC>);
  if (kq <= 2) return pick(local_estimate_kernel<NL, 2, PREC>);
  if (kq <= 6) return pick(local_estimate_kernel<NL, 6, PREC>);
  if (kq <= 24) return pick(local_estimate_kernel<NL, 24, PREC>);
  return LEAD_EINVAL;
}

}  // namespace

// The min-sum kernel (Phase 3) on one side. Its prior: per-qubit LLRs lam_in (shots x n) when
// given, else the merged local posteriors of `table` (use_lead; with the class tables that follow
// the table when `classes` is set), else the channel LLR.
int launch_bp(const lead_code* code, const lead_decode_opts* o, const uint32_t* syn, int64_t shots,
              uint32_t* corr, uint8_t* status, int32_t* iters, float* llr, const float* table,
              cudaStream_t stream, const float* lam_in, void* classes) {
  BPJitArgs a{};
  a.n = code->n;
  a.words_n = code->words_n;
  a.words_m = code->side[o->side].params.words_m;
  a.spb = code->side[o->side].bp_spb;
  a.order = code->order;
  a.max_iter = o->max_iter;
  a.use_lead = o->use_lead ? 1 : 0;
  a.alpha = o->alpha;
  a.p = (float)o->p;
  a.shots = shots;
  a.syn = syn;
  a.corr = corr;
  a.status = status;
  a.iters = iters;
  a.llr = llr;
  a.table = table;
  if (table && classes) {
    const ClassTables ct = class_tables(code, o->side, classes);
    a.cls = ct.cls;
    a.pair = reinterpret_cast<const float*>(ct.pair);
    a.header = ct.header;
  }
  a.lam = lam_in;
  a.pa = code->dside[o->side].bp_pa;
  a.views = code->dside[o->side].views;
  a.check = code->d_check;
  if (!a.pa) return LEAD_EINVAL;
  return jit_launch_bp(code, o->side, o->precision, a, sm_count(code->device), stream);
}

}  // namespace lead

extern "C" {

size_t lead_workspace_bytes(const lead_code* code, const lead_decode_opts* opts, int64_t shots) {
  (void)shots;
  if (!code || !opts || opts->side < 0 || opts->side > 1) return 0;
  // the local posterior table, then (lead_local_estimate) its class bytes and pair table
  return opts->use_lead ? lead::table_bytes(code, opts->side) + lead::local_pair_extra_bytes(code, opts->side) : 0;
}

int lead_local_estimate(const lead_code* code, const lead_decode_opts* opts, const uint32_t* syn,
                        int64_t shots, void* llr, void* workspace, size_t ws_bytes, void* stream) {
  using namespace lead;
  int rc = check_device(code);
  if (rc != LEAD_OK) return rc;
  rc = validate_opts(code, opts);
  if (rc != LEAD_OK) return rc;
  if (shots < 0) return LEAD_EINVAL;
  if (shots == 0) return LEAD_OK;          // empty batch: nothing to read or write
  if (!syn || !llr || !workspace) return LEAD_EINVAL;
  const size_t tb = table_bytes(code, opts->side);
  if (((uintptr_t)workspace & 15) || ws_bytes < tb + local_pair_extra_bytes(code, opts->side)) return LEAD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  float* table = static_cast<float*>(workspace);
  rc = launch_table(code, opts->side, opts->p, table, s, opts->estimator, nullptr);
  if (rc != LEAD_OK) return rc;
  rc = launch_local_pair(code, opts, syn, shots, llr, table, static_cast<char*>(workspace) + tb, s);
  if (rc == LEAD_OK) return check_result(code, stream);
  if (rc != LEAD_EINVAL) return rc;
  // codes the packed view coordinates cannot describe: the direct evaluation per qubit
  auto go = [&](auto prec) -> int {
    constexpr int PR = decltype(prec)::value;
    if (code->nl == 16) return launch_local<16, PR>(code, opts, syn, shots, llr, table, s);
    return launch_local<36, PR>(code, opts, syn, shots, llr, table, s);
  };
  if (opts->precision == LEAD_PREC_BF16) rc = go(std::integral_constant<int, LEAD_PREC_BF16>{});
  else if (opts->precision == LEAD_PREC_FP16) rc = go(std::integral_constant<int, LEAD_PREC_FP16>{});
  else rc = go(std::integral_constant<int, LEAD_PREC_FP32>{});
  return rc == LEAD_OK ? check_result(code, stream) : rc;
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
  void* classes = nullptr;
  if (opts->use_lead) {
    if (!workspace || ((uintptr_t)workspace & 15) || ws_bytes < decode_workspace_bytes(code, opts->side))
      return LEAD_EINVAL;
    table = static_cast<float*>(workspace);
    classes = static_cast<char*>(workspace) + table_bytes(code, opts->side);
    rc = launch_table(code, opts->side, opts->p, table, s, opts->estimator, nullptr);
    if (rc != LEAD_OK) return rc;
    rc = launch_classify(code, opts->side, opts->alpha, LEAD_PREC_FP32, table, classes, s);
    if (rc != LEAD_OK) return rc;
  }
  rc = launch_bp(code, opts, syn, shots, corr, status, iters, llr, table, s, nullptr, classes);
  return rc == LEAD_OK ? check_result(code, stream) : rc;
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
static_assert(LEAD_NOALLOC_TABLE_BYTES % 256 == 0, "scratch must be a whole number of 256-byte blocks");

// Shared by every call on a device and kept until the process exits; holds the last call's
// local posterior table followed by its class tables.
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
  if (shots == 0) return LEAD_OK;          // empty batch: nothing to read or write (as lead_decode)
  if (!syn || !corr || !status) return LEAD_EINVAL;
  if (opts->use_lead && decode_workspace_bytes(code, opts->side) > (size_t)LEAD_NOALLOC_TABLE_BYTES)
    return LEAD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  float* table = nullptr;
  void* classes = nullptr;
  if (opts->use_lead) {
    rc = noalloc_table(code->device, &table);
    if (rc != LEAD_OK) return rc;
    classes = reinterpret_cast<char*>(table) + table_bytes(code, opts->side);
    rc = launch_table(code, opts->side, opts->p, table, s, opts->estimator, nullptr);
    if (rc != LEAD_OK) return rc;
    rc = launch_classify(code, opts->side, opts->alpha, LEAD_PREC_FP32, table, classes, s);
    if (rc != LEAD_OK) return rc;
  }
  rc = launch_bp(code, opts, syn, shots, corr, status, iters, llr, table, s, nullptr, classes);
  return rc == LEAD_OK ? check_result(code, stream) : rc;
}
