// Iterated LEAD: Algorithm 1 run again, with per-qubit priors taken from the global posterior,
// on the shots whose global min-sum did not converge. The paper runs Algorithm 1 once; this is
// an extension built from its parts:
//   round 0: lead_decode (Phases 1-3 with the channel prior);
//   round r >= 1: for the shots without LEAD_ST_CONVERGED, p_i = 1 / (1 + e^{post_i}) from the
//     previous round's posterior LLR (flip_prob_f32, binary32), then
//     lead_decode_priors (Phase 1 as the exact local posterior under those priors, Phase 2,
//     Phase 3) on a compacted batch, and the results scattered back.
// Kernels here: the ordered compaction of unconverged shots, the gather (syndromes + priors) and
// the scatter. All three are HBM-bound copies; the decode calls dominate.

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lead_device.cuh"

namespace lead {
namespace {

constexpr int kMaxRounds = 64;
constexpr int kSelectThreads = 1024;

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// p = 1 / (1 + e^x), the flip probability of a posterior LLR x, in binary32 with every operation
// rounded to nearest (no contraction): x clamped to [-17, 17] (beyond it p lies outside
// [2^-23, 1 - 2^-23], where the per-qubit prior is clamped anyway); k = rint(x / ln 2);
// r = (x - k LN2_HI) - k LN2_LO with LN2_HI = 0.693359375 (9 significant bits: k LN2_HI is exact
// for |k| <= 25); e^r by its Taylor series through r^7 in Horner form; e^x = e^r 2^k (exact).
// Each constant is its binary64 value rounded once to binary32.
__device__ __forceinline__ float flip_prob_f32(float x) {
  constexpr float kInvLn2 = (float)1.4426950408889634;
  constexpr float kLn2Hi = 0.693359375f;
  constexpr float kLn2Lo = (float)(0.6931471805599453 - 0.693359375);
  constexpr float kInvFact[8] = {(float)(1.0 / 1.0),  (float)(1.0 / 1.0),   (float)(1.0 / 2.0),
                                 (float)(1.0 / 6.0),  (float)(1.0 / 24.0),  (float)(1.0 / 120.0),
                                 (float)(1.0 / 720.0), (float)(1.0 / 5040.0)};
  x = fminf(fmaxf(x, -17.0f), 17.0f);
  const float k = rintf(__fmul_rn(x, kInvLn2));
  const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(k, kLn2Hi)), __fmul_rn(k, kLn2Lo));
  float s = kInvFact[7];
#pragma unroll
  for (int n = 6; n >= 0; --n) s = __fadd_rn(__fmul_rn(s, r), kInvFact[n]);
  const float e = __fmul_rn(s, __int_as_float(((int)k + 127) << 23));
  return __fdiv_rn(1.0f, __fadd_rn(1.0f, e));
}

// Indices of the shots whose status lacks LEAD_ST_CONVERGED, in increasing order, and their
// number. One CTA walks the batch 1024 shots at a time: a ballot per warp, the 32 warp counts
// summed in shared memory, each picked shot written at its rank.
__global__ void __launch_bounds__(kSelectThreads) select_unconverged_kernel(const uint8_t* __restrict__ status,
                                                                            int64_t shots, int32_t* __restrict__ list,
                                                                            int32_t* __restrict__ count) {
  __shared__ int warp_n[kSelectThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int base = 0;
  for (int64_t s0 = 0; s0 < shots; s0 += kSelectThreads) {
    const int64_t s = s0 + threadIdx.x;
    const bool pick = s < shots && !(status[s] & LEAD_ST_CONVERGED);
    const unsigned int b = __ballot_sync(0xFFFFFFFFu, pick);
    if (lane == 0) warp_n[warp] = __popc(b);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll 8
    for (int w = 0; w < kSelectThreads / 32; ++w) {
      const int c = warp_n[w];
      before += w < warp ? c : 0;
      total += c;
    }
    if (pick) list[base + before + __popc(b & ((1u << lane) - 1u))] = (int32_t)s;
    base += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

// Compacted inputs of the next round: row j takes shot list[j]'s syndrome and, per qubit, the
// prior p = flip_prob_f32(post) of that shot's last posterior LLR.
__global__ void iter_gather_kernel(const int32_t* __restrict__ list, int64_t cnt, const uint32_t* __restrict__ syn,
                                   int wm, const float* __restrict__ post, int n, uint32_t* __restrict__ syn_c,
                                   float* __restrict__ prior_c) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t t = t0; t < cnt * wm; t += stride) {
    const int64_t j = t / wm;
    syn_c[t] = syn[(int64_t)list[j] * wm + (t - j * wm)];
  }
  for (int64_t t = t0; t < cnt * n; t += stride) {
    const int64_t j = t / n;
    prior_c[t] = flip_prob_f32(post[(int64_t)list[j] * n + (t - j * n)]);
  }
}

// Results of the compacted round back into the caller's rows: correction, status, posterior,
// and the round's iterations added to the shot's total.
__global__ void iter_scatter_kernel(const int32_t* __restrict__ list, int64_t cnt, const uint32_t* __restrict__ corr_c,
                                    const uint8_t* __restrict__ st_c, const int32_t* __restrict__ it_c,
                                    const float* __restrict__ post_c, int wn, int n, uint32_t* __restrict__ corr,
                                    uint8_t* __restrict__ status, int32_t* __restrict__ iters,
                                    float* __restrict__ post) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t t = t0; t < cnt; t += stride) {
    const int64_t s = list[t];
    status[s] = st_c[t];
    if (iters) iters[s] += it_c[t];
  }
  for (int64_t t = t0; t < cnt * wn; t += stride) {
    const int64_t j = t / wn;
    corr[(int64_t)list[j] * wn + (t - j * wn)] = corr_c[t];
  }
  for (int64_t t = t0; t < cnt * n; t += stride) {
    const int64_t j = t / n;
    post[(int64_t)list[j] * n + (t - j * n)] = post_c[t];
  }
}

// Workspace regions, each starting on a 256-byte boundary: the inner decode workspace first
// (lead_decode and lead_decode_priors both use it), then the compaction list and its count, the
// compacted syndromes, priors (overwritten by the round's posteriors), corrections, statuses
// and iterations.
struct IterLayout {
  size_t inner, list, count, syn, prior, corr, st, it, total;
};

IterLayout iter_layout(const lead_code* code, const lead_decode_opts* o, int64_t shots) {
  IterLayout L{};
  const int wm = code->side[o->side].params.words_m;
  size_t off = round256(std::max(lead_workspace_bytes(code, o, shots), lead_priors_workspace_bytes(code, o, shots)));
  L.inner = 0;
  L.list = off;
  off += round256((size_t)shots * 4);
  L.count = off;
  off += 256;
  L.syn = off;
  off += round256((size_t)shots * wm * 4);
  L.prior = off;
  off += round256((size_t)shots * code->n * 4);
  L.corr = off;
  off += round256((size_t)shots * code->words_n * 4);
  L.st = off;
  off += round256((size_t)shots);
  L.it = off;
  off += round256((size_t)shots * 4);
  L.total = off;
  return L;
}

unsigned int copy_grid(const lead_code* code, int64_t elems) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((elems + 255) / 256, (int64_t)sm_count(code->device) * 8));
  return (unsigned int)blocks;
}

}  // namespace
}  // namespace lead

extern "C" {

size_t lead_iterated_workspace_bytes(const lead_code* code, const lead_decode_opts* opts, int64_t shots) {
  if (!code || !opts || shots < 0 || opts->side < 0 || opts->side > 1) return 0;
  return lead::iter_layout(code, opts, shots).total;
}

int lead_decode_iterated(const lead_code* code, const lead_decode_opts* opts, int32_t rounds, const uint32_t* syn,
                         int64_t shots, uint32_t* corr, uint8_t* status, int32_t* iters, float* llr,
                         void* workspace, size_t ws_bytes, void* stream) {
  using namespace lead;
  if (!code || !opts || opts->side < 0 || opts->side > 1) return LEAD_EINVAL;
  if (rounds < 1 || rounds > kMaxRounds || shots < 0 || shots > INT32_MAX) return LEAD_EINVAL;
  if (shots == 0) return LEAD_OK;
  if (!syn || !corr || !status || !workspace || ((uintptr_t)workspace & 255)) return LEAD_EINVAL;
  if (rounds > 1 && !llr) return LEAD_EINVAL;
  const IterLayout Ly = iter_layout(code, opts, shots);
  if (ws_bytes < Ly.total) return LEAD_EINVAL;
  lead_decode_opts po = *opts;
  po.estimator = LEAD_EST_EXACT;                 // per-qubit priors: the exact local posterior
  int rc = rounds > 1 ? priors_check(code, &po) : LEAD_OK;
  if (rc != LEAD_OK) return rc;
  char* ws = static_cast<char*>(workspace);
  cudaStream_t s = (cudaStream_t)stream;
  // round 0: Algorithm 1 with the channel prior
  rc = lead_decode(code, opts, syn, shots, corr, status, iters, llr, ws + Ly.inner, Ly.list, stream);
  if (rc != LEAD_OK) return rc;
  int32_t* list = reinterpret_cast<int32_t*>(ws + Ly.list);
  int32_t* d_count = reinterpret_cast<int32_t*>(ws + Ly.count);
  uint32_t* syn_c = reinterpret_cast<uint32_t*>(ws + Ly.syn);
  float* prior_c = reinterpret_cast<float*>(ws + Ly.prior);
  uint32_t* corr_c = reinterpret_cast<uint32_t*>(ws + Ly.corr);
  uint8_t* st_c = reinterpret_cast<uint8_t*>(ws + Ly.st);
  int32_t* it_c = reinterpret_cast<int32_t*>(ws + Ly.it);
  const int wm = code->side[opts->side].params.words_m, wn = code->words_n, n = code->n;
  for (int r = 1; r < rounds; ++r) {
    select_unconverged_kernel<<<1, kSelectThreads, 0, s>>>(status, shots, list, d_count);
    LEAD_CUDA_TRY(cudaGetLastError());
    int32_t cnt = 0;
    LEAD_CUDA_TRY(cudaMemcpyAsync(&cnt, d_count, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    LEAD_CUDA_TRY(cudaStreamSynchronize(s));
    if (cnt == 0) break;
    iter_gather_kernel<<<copy_grid(code, (int64_t)cnt * n), 256, 0, s>>>(list, cnt, syn, wm, llr, n, syn_c, prior_c);
    LEAD_CUDA_TRY(cudaGetLastError());
    // prior_c doubles as the posterior output: each pass of lead_decode_priors turns its rows'
    // priors into prior LLRs in the inner workspace before its min-sum writes those rows.
    rc = lead_decode_priors(code, &po, syn_c, cnt, prior_c, corr_c, st_c, it_c, prior_c, ws + Ly.inner, Ly.list,
                            stream);
    if (rc != LEAD_OK) return rc;
    iter_scatter_kernel<<<copy_grid(code, (int64_t)cnt * n), 256, 0, s>>>(list, cnt, corr_c, st_c, it_c, prior_c, wn,
                                                                           n, corr, status, iters, llr);
    LEAD_CUDA_TRY(cudaGetLastError());
  }
  return check_result(code, stream);
}

}  // extern "C"
