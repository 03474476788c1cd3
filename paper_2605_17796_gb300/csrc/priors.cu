// Phase 1 with per-qubit (non-uniform) priors: the exact local posterior of every (shot, vertex)
// under the product of its qubits' own priors, evaluated per item by the row grouping of the
// local check matrix L = kron(R_B, R_A):
//   * row a of the local view is a pattern x of Delta bits with log-weight -sum_b x_b w_ab
//     (w = lambda(p), the prior LLR) relative to the all-zero row; its image f = R_B x is one of
//     2^kB classes; R_a(f) = log sum of the class, rho_ab(f) = share of the class with x_b = 1;
//   * the row images F = (f_a) consistent with the local syndrome form the coset
//     base(s) + kernel(R_A) (2^(Delta kB - m_l) members); L_F = sum_a R_a(f_a);
//   * q_ab = sum_F e^{L_F} rho_ab(f_a(F)) / sum_F e^{L_F}.
// The hard decision is the least integer cost sum_j e_j W_j, W_j = rint(2^20 lambda(p_j)), ties
// by the least row-major key (as the uniform path); the boost raises its bits to 1/2.
// One warp per item; per-warp scratch in shared memory; warp reductions in a fixed order, so
// results are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "bp_jit_args.h"
#include "lead_device.cuh"

namespace lead {
int check_device(const lead_code* code);
int run_prior_local_tc(const lead_code* code, int side, const uint32_t* syn, int64_t shots, const float* lam,
                       float* Q, uint64_t* ml, unsigned int* err, cudaStream_t stream);
int launch_bp(const lead_code* code, const lead_decode_opts* o, const uint32_t* syn, int64_t shots,
              uint32_t* corr, uint8_t* status, int32_t* iters, float* llr, const float* table,
              cudaStream_t stream, const float* lam_in, void* classes);

namespace {

// The local posterior under per-qubit priors runs on the tensor cores (prior_tc.cu). Setting
// LEAD_PRIOR_SIMT=1 in the environment (read at every call) selects the CUDA-core kernel below
// instead (the same reading of Phase 1, one warp per item, both contractions as gathers), so the
// two can be compared on the same inputs.
bool prior_simt() {
  const char* e = std::getenv("LEAD_PRIOR_SIMT");
  return e && e[0] && e[0] != '0';
}

constexpr int kPriorWarps = 8;

struct PriorArgs {
  int n, order, words_m;
  int64_t items;              // shots * order
  const uint32_t* syn;
  const float* prior;         // shots x n
  const uint16_t* views;
  const uint8_t* xcls;        // 2^Delta row patterns, class-major, increasing within a class
  const uint32_t* cbase;      // 2^m_l packed row images
  const uint32_t* ckern;      // NK packed kernel elements
  float* Q;                   // items x nl boosted local posteriors
  unsigned long long* ml;     // items: least-cost local decision (bit j = local index j), or null
};

template <int DELTA, int KB, int ML, int NK>
__global__ void __launch_bounds__(kPriorWarps * 32) prior_local_kernel(PriorArgs a) {
  constexpr int NL = DELTA * DELTA, NX = 1 << DELTA, NF = 1 << KB;
  constexpr int KPL = (NK + 31) / 32;                  // coset members per lane
  constexpr int CS = NX / NF;                          // row patterns per class
  __shared__ float s_w[kPriorWarps][DELTA][DELTA];
  __shared__ int s_W[kPriorWarps][DELTA][DELTA];
  __shared__ float s_logr[kPriorWarps][DELTA][NX];
  __shared__ int s_cost[kPriorWarps][DELTA][NX];
  __shared__ float s_R[kPriorWarps][DELTA][NF];
  __shared__ float s_rho[kPriorWarps][DELTA][DELTA][NF];
  __shared__ int s_cmin[kPriorWarps][DELTA][NF];
  __shared__ unsigned char s_xmin[kPriorWarps][DELTA][NF];
  __shared__ float s_agg[kPriorWarps][DELTA][NF];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * kPriorWarps;
  for (int64_t item = (int64_t)blockIdx.x * kPriorWarps + wid; item < a.items; item += nwarps) {
    const int64_t shot = item / a.order;
    const int v = (int)(item - shot * a.order);
    const uint32_t s = bit_field(a.syn + shot * a.words_m, v * ML, ML);
    // A: prior LLRs and integer costs of the view's positions, stored as [row a][column b]
    for (int j = lane; j < NL; j += 32) {
      const int q = __ldg(a.views + v * NL + j);
      const float w = llr_f32(__ldg(a.prior + shot * a.n + q));
      const int ia = j % DELTA, ib = j / DELTA;
      s_w[wid][ia][ib] = w;
      s_W[wid][ia][ib] = __float2int_rn(__fmul_rn(w, 1048576.0f));
    }
    __syncwarp();
    // B: row patterns
    for (int idx = lane; idx < DELTA * NX; idx += 32) {
      const int ra = idx / NX, x = idx - ra * NX;
      float acc = 0.0f;
      int c = 0;
#pragma unroll
      for (int b = 0; b < DELTA; ++b)
        if ((x >> b) & 1) {
          acc = __fadd_rn(acc, s_w[wid][ra][b]);
          c += s_W[wid][ra][b];
        }
      s_logr[wid][ra][x] = -acc;
      s_cost[wid][ra][x] = c;
    }
    __syncwarp();
    // C: classes of row images (the members of a class in increasing order: the first least
    // cost is the least pattern)
    for (int idx = lane; idx < DELTA * NF; idx += 32) {
      const int ra = idx / NF, f = idx - ra * NF;
      const unsigned char* xs = a.xcls + f * CS;
      float m = -INFINITY;
      int cmin = 0x7FFFFFFF, xmin = 0;
#pragma unroll
      for (int t = 0; t < CS; ++t) {
        const int x = __ldg(xs + t);
        m = fmaxf(m, s_logr[wid][ra][x]);
        const int c = s_cost[wid][ra][x];
        if (c < cmin) {
          cmin = c;
          xmin = x;
        }
      }
      float sum = 0.0f, sb[DELTA];
#pragma unroll
      for (int b = 0; b < DELTA; ++b) sb[b] = 0.0f;
#pragma unroll
      for (int t = 0; t < CS; ++t) {
        const int x = __ldg(xs + t);
        const float e = expf(s_logr[wid][ra][x] - m);
        sum += e;
#pragma unroll
        for (int b = 0; b < DELTA; ++b)
          if ((x >> b) & 1) sb[b] += e;
      }
      s_R[wid][ra][f] = m + logf(sum);
#pragma unroll
      for (int b = 0; b < DELTA; ++b) s_rho[wid][ra][b][f] = sb[b] / sum;
      s_cmin[wid][ra][f] = cmin;
      s_xmin[wid][ra][f] = (unsigned char)xmin;
    }
    __syncwarp();
    // D: the coset of row images; lane l takes members l, l + 32, ...
    const uint32_t base = __ldg(a.cbase + s);
    uint32_t Fm[KPL];
    float em[KPL];
    float lmax = -INFINITY;
    long long best_cost = 0x7FFFFFFFFFFFFFFFll;
    unsigned long long best_key = ~0ull;
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      const int i = lane + 32 * t;
      const bool ok = i < NK;
      const uint32_t F = base ^ (ok ? __ldg(a.ckern + i) : 0u);
      float L = 0.0f;
      long long c = 0;
      unsigned long long key = 0;
#pragma unroll
      for (int ra = 0; ra < DELTA; ++ra) {
        const int f = (F >> (ra * KB)) & (NF - 1);
        L = __fadd_rn(L, s_R[wid][ra][f]);
        c += s_cmin[wid][ra][f];
        key |= (unsigned long long)s_xmin[wid][ra][f] << (ra * DELTA);
      }
      Fm[t] = F;
      em[t] = ok ? L : -INFINITY;
      lmax = fmaxf(lmax, em[t]);
      if (ok && (c < best_cost || (c == best_cost && key < best_key))) {
        best_cost = c;
        best_key = key;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lmax = fmaxf(lmax, __shfl_xor_sync(0xFFFFFFFFu, lmax, o));
      const long long oc = __shfl_xor_sync(0xFFFFFFFFu, best_cost, o);
      const unsigned long long ok = __shfl_xor_sync(0xFFFFFFFFu, best_key, o);
      if (oc < best_cost || (oc == best_cost && ok < best_key)) {
        best_cost = oc;
        best_key = ok;
      }
    }
    float Z = 0.0f;
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      em[t] = expf(em[t] - lmax);                      // 0 for the padding members
      Z += em[t];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Z += __shfl_xor_sync(0xFFFFFFFFu, Z, o);
    // class sums agg[a][f] = sum of e^(L_F - max) over the members with f_a(F) = f, row by row
#pragma unroll 1
    for (int ra = 0; ra < DELTA; ++ra) {
      float ag[NF];
#pragma unroll
      for (int g = 0; g < NF; ++g) ag[g] = 0.0f;
#pragma unroll
      for (int t = 0; t < KPL; ++t) {
        const int f = (Fm[t] >> (ra * KB)) & (NF - 1);
#pragma unroll
        for (int g = 0; g < NF; ++g) ag[g] += (f == g) ? em[t] : 0.0f;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int g = 0; g < NF; ++g) ag[g] += __shfl_xor_sync(0xFFFFFFFFu, ag[g], o);
      if (lane == 0) {
#pragma unroll
        for (int g = 0; g < NF; ++g) s_agg[wid][ra][g] = ag[g];
      }
    }
    __syncwarp();
    // E: marginals, boost by the least-cost member, store
    if (a.ml && lane == 0) {
      unsigned long long mask = 0;
#pragma unroll
      for (int ra = 0; ra < DELTA; ++ra)
#pragma unroll
        for (int b = 0; b < DELTA; ++b)
          mask |= ((best_key >> (ra * DELTA + b)) & 1ull) << (b * DELTA + ra);
      a.ml[item] = mask;
    }
    for (int j = lane; j < NL; j += 32) {
      const int ia = j % DELTA, ib = j / DELTA;
      float num = 0.0f;
#pragma unroll
      for (int f = 0; f < NF; ++f) num += s_agg[wid][ia][f] * s_rho[wid][ia][ib][f];
      float q = num / Z;
      const int xrow = (int)((best_key >> (ia * DELTA)) & (NX - 1));
      if ((xrow >> ib) & 1) q = fmaxf(q, 0.5f);
      a.Q[item * NL + j] = q;
    }
    __syncwarp();
  }
}

struct MergeArgs {
  int n, order, nl;
  int64_t shots;
  float alpha;
  const float* Q;
  const uint32_t* qslots;
  float* llr;
};

// Phase 2 on the boosted local posteriors: the two views of every qubit are merged into its LLR.
__global__ void prior_merge_kernel(MergeArgs a) {
  const int64_t total = a.shots * a.n;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t shot = idx / a.n;
    const int i = (int)(idx - shot * a.n);
    const uint32_t s0 = __ldg(a.qslots + 2 * i), s1 = __ldg(a.qslots + 2 * i + 1);
    const float* Qs = a.Q + shot * (int64_t)a.order * a.nl;
    a.llr[idx] = merged_llr(Qs[s0], Qs[s1], a.alpha);
  }
}

// The standalone baseline with per-qubit priors: lambda(p_i) for every qubit.
__global__ void prior_channel_kernel(int64_t total, const float* prior, float* llr) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x)
    llr[idx] = llr_f32(__ldg(prior + idx));
}

template <int DELTA, int KB, int ML, int NK>
int launch_prior_local(const lead_code* code, int side, const uint32_t* syn, int64_t shots, const float* prior,
                       float* Q, uint64_t* ml, cudaStream_t stream) {
  const DeviceSide& ds = code->dside[side];
  PriorArgs a{};
  a.n = code->n;
  a.order = code->order;
  a.words_m = code->side[side].params.words_m;
  a.items = shots * code->order;
  a.syn = syn;
  a.prior = prior;
  a.views = ds.views;
  a.xcls = ds.xcls;
  a.cbase = ds.cbase;
  a.ckern = ds.ckern;
  a.Q = Q;
  a.ml = reinterpret_cast<unsigned long long*>(ml);
  const int64_t blocks = std::min<int64_t>((a.items + kPriorWarps - 1) / kPriorWarps,
                                           (int64_t)sm_count(code->device) * 16);
  prior_local_kernel<DELTA, KB, ML, NK><<<(unsigned)blocks, kPriorWarps * 32, 0, stream>>>(a);
  LEAD_CUDA_TRY(cudaGetLastError());
  return LEAD_OK;
}

// Supported local codes: the kernel is instantiated per (Delta, k_B, m_l); other shapes report
// LEAD_EINVAL.
int run_prior_local(const lead_code* code, int side, const uint32_t* syn, int64_t shots, const float* prior,
                    float* Q, uint64_t* ml, cudaStream_t stream) {
  const HostSide& hs = code->side[side];
  const DeviceSide& ds = code->dside[side];
  if (!ds.xcls || !ds.cbase || !ds.ckern) return LEAD_EINVAL;
  const size_t nk = hs.ckern.size();
  if (code->delta == 6 && hs.kRB == 3 && hs.m_l == 9 && nk == 512)
    return launch_prior_local<6, 3, 9, 512>(code, side, syn, shots, prior, Q, ml, stream);
  if (code->delta == 4 && hs.kRB == 2 && hs.m_l == 4 && nk == 16)
    return launch_prior_local<4, 2, 4, 16>(code, side, syn, shots, prior, Q, ml, stream);
  return LEAD_EINVAL;
}

int run_prior_llr(const lead_code* code, const lead_decode_opts* o, const uint32_t* syn, int64_t shots,
                  const float* prior, float* llr, float* Q, uint64_t* ml, cudaStream_t stream) {
  // lambda(p_i) for every qubit: the baseline's prior, and with the local stage the input of the
  // local posterior kernel (the merge below then overwrites it with the merged LLRs)
  const int64_t total = shots * code->n;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)sm_count(code->device) * 8);
  prior_channel_kernel<<<(unsigned)blocks, 256, 0, stream>>>(total, prior, llr);
  LEAD_CUDA_TRY(cudaGetLastError());
  if (!o->use_lead) return LEAD_OK;
  int rc = prior_simt() ? run_prior_local(code, o->side, syn, shots, prior, Q, ml, stream)
                        : run_prior_local_tc(code, o->side, syn, shots, llr, Q, ml,
                                             reinterpret_cast<unsigned int*>(code->d_check + 4), stream);
  if (rc != LEAD_OK) return rc;
  MergeArgs m{};
  m.n = code->n;
  m.order = code->order;
  m.nl = code->nl;
  m.shots = shots;
  m.alpha = o->alpha;
  m.Q = Q;
  m.qslots = code->dside[o->side].qslots;
  m.llr = llr;
  prior_merge_kernel<<<(unsigned)blocks, 256, 0, stream>>>(m);
  LEAD_CUDA_TRY(cudaGetLastError());
  return LEAD_OK;
}

size_t q_bytes(const lead_code* code, int64_t shots) {
  return ((size_t)shots * code->order * code->nl * sizeof(float) + 255) / 256 * 256;
}
size_t lam_bytes(const lead_code* code, int64_t shots) {
  return ((size_t)shots * code->n * sizeof(float) + 255) / 256 * 256;
}

// Shots per pass: the local posteriors and prior LLRs of one pass fit in about 256 MiB.
constexpr size_t kPriorPassBytes = size_t(256) << 20;
int64_t pass_shots(const lead_code* code, int64_t shots) {
  const size_t per_shot = (size_t)code->order * code->nl * sizeof(float) + (size_t)code->n * sizeof(float);
  return std::max<int64_t>(1, std::min<int64_t>(shots, (int64_t)(kPriorPassBytes / per_shot)));
}

int validate(const lead_code* code, const lead_decode_opts* o) {
  if (!o || o->side < 0 || o->side > 1 || o->max_iter < 0 || o->max_iter > kMaxIter) return LEAD_EINVAL;
  if (!(o->alpha > 0.0f && o->alpha <= 1.0f) || o->precision < 0 || o->precision >= kPrecModes) return LEAD_EINVAL;
  if (o->estimator != LEAD_EST_EXACT) return LEAD_EINVAL;     // per-qubit priors: exact posterior only
  return LEAD_OK;
}

}  // namespace

// The checks lead_decode_priors makes before any device work: device, options and, with the
// local stage, a local code the per-qubit kernel serves.
int priors_check(const lead_code* code, const lead_decode_opts* o) {
  int rc = check_device(code);
  if (rc != LEAD_OK) return rc;
  rc = validate(code, o);
  if (rc != LEAD_OK || !o->use_lead) return rc;
  const HostSide& hs = code->side[o->side];
  const DeviceSide& ds = code->dside[o->side];
  if (!ds.xcls || !ds.cbase || !ds.ckern) return LEAD_EINVAL;
  const size_t nk = hs.ckern.size();
  const bool ok = (code->delta == 6 && hs.kRB == 3 && hs.m_l == 9 && nk == 512) ||
                  (code->delta == 4 && hs.kRB == 2 && hs.m_l == 4 && nk == 16);
  return ok ? LEAD_OK : LEAD_EINVAL;
}

}  // namespace lead

extern "C" {

size_t lead_priors_workspace_bytes(const lead_code* code, const lead_decode_opts* opts, int64_t shots) {
  if (!code || !opts || shots < 0) return 0;
  const int64_t c = lead::pass_shots(code, shots);
  return lead::q_bytes(code, c) + lead::lam_bytes(code, c);
}

int lead_local_estimate_priors(const lead_code* code, const lead_decode_opts* opts, const uint32_t* syn,
                               int64_t shots, const float* prior, float* llr, float* q_out, uint64_t* ml_out,
                               void* workspace, size_t ws_bytes, void* stream) {
  using namespace lead;
  int rc = check_device(code);
  if (rc != LEAD_OK) return rc;
  rc = validate(code, opts);
  if (rc != LEAD_OK) return rc;
  if (shots < 0) return LEAD_EINVAL;
  if (shots == 0) return LEAD_OK;
  if (!syn || !prior || !llr) return LEAD_EINVAL;
  const int64_t chunk = q_out ? shots : pass_shots(code, shots);
  if (!q_out && (!workspace || ((uintptr_t)workspace & 15) || ws_bytes < q_bytes(code, chunk)))
    return LEAD_EINVAL;
  lead_decode_opts o = *opts;
  o.use_lead = 1;
  const int wm = code->side[o.side].params.words_m, n = code->n;
  const int64_t per_item = (int64_t)code->order * code->nl;
  for (int64_t c0 = 0; c0 < shots; c0 += chunk) {
    const int64_t cn = std::min(chunk, shots - c0);
    float* Q = q_out ? q_out + c0 * per_item : static_cast<float*>(workspace);
    rc = run_prior_llr(code, &o, syn + c0 * wm, cn, prior + c0 * n, llr + c0 * n, Q,
                       ml_out ? ml_out + c0 * code->order : nullptr, (cudaStream_t)stream);
    if (rc != LEAD_OK) return rc;
  }
  return check_result(code, stream);
}

int lead_decode_priors(const lead_code* code, const lead_decode_opts* opts, const uint32_t* syn, int64_t shots,
                       const float* prior, uint32_t* corr, uint8_t* status, int32_t* iters, float* llr,
                       void* workspace, size_t ws_bytes, void* stream) {
  using namespace lead;
  int rc = check_device(code);
  if (rc != LEAD_OK) return rc;
  rc = validate(code, opts);
  if (rc != LEAD_OK) return rc;
  if (shots < 0) return LEAD_EINVAL;
  if (shots == 0) return LEAD_OK;
  if (!syn || !prior || !corr || !status) return LEAD_EINVAL;
  const int64_t chunk = pass_shots(code, shots);
  if (!workspace || ((uintptr_t)workspace & 15) || ws_bytes < q_bytes(code, chunk) + lam_bytes(code, chunk))
    return LEAD_EINVAL;
  float* Q = static_cast<float*>(workspace);
  float* lam = reinterpret_cast<float*>(static_cast<char*>(workspace) + q_bytes(code, chunk));
  cudaStream_t s = (cudaStream_t)stream;
  const int wm = code->side[opts->side].params.words_m, n = code->n, wn = code->words_n;
  for (int64_t c0 = 0; c0 < shots; c0 += chunk) {
    const int64_t cn = std::min(chunk, shots - c0);
    rc = run_prior_llr(code, opts, syn + c0 * wm, cn, prior + c0 * n, lam, Q, nullptr, s);
    if (rc != LEAD_OK) return rc;
    rc = launch_bp(code, opts, syn + c0 * wm, cn, corr + c0 * wn, status + c0, iters ? iters + c0 : nullptr,
                   llr ? llr + c0 * n : nullptr, nullptr, s, lam, nullptr);
    if (rc != LEAD_OK) return rc;
  }
  return check_result(code, stream);
}

}  // extern "C"
