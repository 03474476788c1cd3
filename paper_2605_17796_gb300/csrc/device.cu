// Device tables of a code, the exact local coset enumerators (Phase 1, p-independent part) and
// the per-p local posterior table (Phase 1 + boost).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "lead_device.cuh"

namespace lead {

std::vector<uint16_t> single_cta_partner_table(const lead_code* code, int side, const Geometry& g) {
  const HostSide& hs = code->side[side];
  const int nl = code->nl;
  std::vector<uint16_t> pa((size_t)nl * g.ts, 0);
  for (int sl = 0; sl < g.spb; ++sl)
    for (int v = 0; v < code->order; ++v)
      for (int j = 0; j < nl; ++j) {
        const uint32_t raw = hs.partner[(size_t)v * nl + j];
        const uint32_t ps = raw & 0x7FFFFFFFu;
        const uint32_t vp = ps / nl, jp = ps % nl;
        const int t = sl * code->order + v;
        pa[(size_t)j * g.ts + t] = (uint16_t)((jp * g.ts + sl * code->order + vp) | ((raw >> 31) << 15));
      }
  return pa;
}

std::vector<uint8_t> partner_table_bytes(const lead_code* code, int side, const Geometry& g) {
  const HostSide& hs = code->side[side];
  const int nl = code->nl;
  std::vector<uint8_t> out;
  auto as_bytes = [&](const auto& v) {
    out.resize(v.size() * sizeof(v[0]));
    std::memcpy(out.data(), v.data(), out.size());
  };
  if (g.cluster == 1) {
    if ((size_t)nl * g.ts < 32768) as_bytes(single_cta_partner_table(code, side, g));
    return out;
  }
  const bool pa16 = cluster_pa16(g, nl);
  std::vector<uint16_t> p16(pa16 ? (size_t)nl * code->order : 0, 0);
  std::vector<uint32_t> p32(pa16 ? 0 : (size_t)nl * code->order, 0);
  for (int v = 0; v < code->order; ++v)
    for (int j = 0; j < nl; ++j) {
      const uint32_t raw = hs.partner[(size_t)v * nl + j];
      const uint32_t ps = raw & 0x7FFFFFFFu;
      const uint32_t vp = ps / nl, jp = ps % nl;
      const uint32_t owner = vp / g.ts, tp = vp - owner * g.ts;
      if (pa16) p16[(size_t)j * code->order + v] = (uint16_t)((jp * g.ts + tp) | (owner << 13) | ((raw >> 31) << 15));
      else p32[(size_t)j * code->order + v] = (jp * g.ts + tp) | (owner << 16) | (raw & 0x80000000u);
    }
  if (pa16) as_bytes(p16);
  else as_bytes(p32);
  return out;
}



int sm_count(int device) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

namespace {

// Row-by-row dynamic programme over the Delta rows of the local view E (rows a, columns b,
// local index j = b*Delta + a). A row pattern x (bit b = E[a][b]) adds contrib[a][x] to the
// local syndrome. Run 0 counts all patterns per (syndrome, weight): N. Run 1 + j counts those
// with bit j set, by admitting at row a = j mod Delta only patterns with bit b = j div Delta.
// State counts stay below 2^36 (64-bit accumulators); final entries are at most 2^(nl - m_l).
__global__ void enumerate_kernel(int delta, int m_l, const uint16_t* __restrict__ contrib,
                                 unsigned long long* __restrict__ bufs, int32_t* __restrict__ N,
                                 int32_t* __restrict__ N1) {
  const int run = blockIdx.x;
  const int nl = delta * delta;
  const int W = nl + 1;
  const int states = 1 << m_l;
  const size_t sz = (size_t)states * W;
  unsigned long long* cur = bufs + (size_t)run * 2 * sz;
  unsigned long long* nxt = cur + sz;
  for (size_t i = threadIdx.x; i < sz; i += blockDim.x) cur[i] = (i == 0) ? 1ull : 0ull;
  __syncthreads();
  const int fj = run - 1;
  for (int a = 0; a < delta; ++a) {
    const int forced_b = (fj >= 0 && fj % delta == a) ? fj / delta : -1;
    const uint16_t* ca = contrib + a * (1 << delta);
    for (size_t i = threadIdx.x; i < sz; i += blockDim.x) {
      const int S = (int)(i / W), w = (int)(i % W);
      unsigned long long acc = 0;
      for (int x = 0; x < (1 << delta); ++x) {
        if (forced_b >= 0 && !((x >> forced_b) & 1)) continue;
        const int wx = __popc(x);
        if (wx > w) continue;
        acc += cur[(size_t)(S ^ ca[x]) * W + (w - wx)];
      }
      nxt[i] = acc;
    }
    __syncthreads();
    unsigned long long* t = cur;
    cur = nxt;
    nxt = t;
  }
  for (size_t i = threadIdx.x; i < sz; i += blockDim.x) {
    const int S = (int)(i / W), w = (int)(i % W);
    const int32_t val = (int32_t)cur[i];
    if (run == 0) N[i] = val;
    else N1[((size_t)S * nl + fj) * W + w] = val;
  }
}

// Least (weight, row-major key) member of every coset by the same row recursion in the
// (min, +) semiring: key = sum_a x_a 2^(a*Delta), packed with the weight as weight<<40 | key;
// comparing packed values compares (weight, key) lexicographically, and the order of partial
// solutions reaching a state is preserved by any common completion.
__global__ void ml_kernel(int delta, int m_l, const uint16_t* __restrict__ contrib,
                          unsigned long long* __restrict__ buf, uint64_t* __restrict__ ml) {
  const int states = 1 << m_l;
  unsigned long long* cur = buf;
  unsigned long long* nxt = buf + states;
  const unsigned long long INF = ~0ull;
  for (int S = threadIdx.x; S < states; S += blockDim.x) cur[S] = (S == 0) ? 0ull : INF;
  __syncthreads();
  for (int a = 0; a < delta; ++a) {
    const uint16_t* ca = contrib + a * (1 << delta);
    for (int S = threadIdx.x; S < states; S += blockDim.x) {
      unsigned long long best = INF;
      for (int x = 0; x < (1 << delta); ++x) {
        const unsigned long long prev = cur[S ^ ca[x]];
        if (prev == INF) continue;
        const unsigned long long cand =
            prev + ((unsigned long long)__popc(x) << 40) + ((unsigned long long)x << (a * delta));
        best = cand < best ? cand : best;
      }
      nxt[S] = best;
    }
    __syncthreads();
    unsigned long long* t = cur;
    cur = nxt;
    nxt = t;
  }
  for (int S = threadIdx.x; S < states; S += blockDim.x) {
    const unsigned long long key = cur[S] & ((1ull << 40) - 1);
    uint64_t mask = 0;
    for (int a = 0; a < delta; ++a)
      for (int b = 0; b < delta; ++b)
        if ((key >> (a * delta + b)) & 1) mask |= 1ull << (b * delta + a);
    ml[S] = cur[S] == INF ? ~0ull : mask;
  }
}

// q[s][j] = N1_s,j(r) / N_s(r), both by Horner from the highest degree with separate binary64
// multiply and add (no fused multiply-add), rounded to binary32; then max(q, 1/2) on the bits
// of the least-weight coset member.
__global__ void table_kernel(int nl, int m_l, double r, const int32_t* __restrict__ N,
                             const int32_t* __restrict__ N1, const uint64_t* __restrict__ ml,
                             float* __restrict__ table) {
  const int W = nl + 1;
  const int total = (1 << m_l) * nl;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int s = i / nl, j = i - s * nl;
    double num = 0.0, den = 0.0;
    for (int w = nl; w >= 0; --w) {
      num = __dadd_rn(__dmul_rn(num, r), (double)N1[((size_t)s * nl + j) * W + w]);
      den = __dadd_rn(__dmul_rn(den, r), (double)N[(size_t)s * W + w]);
    }
    float q = __double2float_rn(__ddiv_rn(num, den));
    if ((ml[s] >> j) & 1) q = fmaxf(q, 0.5f);
    table[i] = q;
  }
}

__global__ void fill_i32_kernel(int32_t* __restrict__ out, int n, int32_t value) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = value;
}

// Phase 1 with local min-sum BP as the LocalDecoder, one thread per local syndrome s: flooding
// min-sum on the vertex's local checks with the binary32 channel LLR on every position and the
// global decoder's rules (c2v = signed minimum over the other positions, sign bits and the
// syndrome bit; U_j = sum of the messages of the rows containing j in increasing row order,
// from 0; post_j = lambda + U_j; e_j = [post_j < 0]; iteration 0 tests the prior; stop at the
// first t with H_v e = s, at most max_iter iterations). q_j = sigmoid(post_j), raised to 1/2 on
// the bits of e when H_v e = s. iters[s] (nullable) = t | converged << 16.
__global__ void minsum_table_kernel(SideParams P, int nl, float p, int max_iter, float* __restrict__ table,
                                    int32_t* __restrict__ iters) {
  const int S = 1 << P.m_l;
  const float lam = channel_llr(p);
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    float post[kMaxDelta * kMaxDelta];
    float c2v[kMaxLocalRows][kMaxSupport];
    for (int j = 0; j < nl; ++j) post[j] = lam;
    for (int r = 0; r < P.m_l; ++r)
      for (int k = 0; k < P.supp_len[r]; ++k) c2v[r][k] = 0.0f;
    bool conv = false;
    int t = 0;
    for (;; ++t) {
      if (t > 0) {
        for (int r = 0; r < P.m_l; ++r) {
          const int L = P.supp_len[r];
          float n1 = __int_as_float(0x7F800000), n2 = __int_as_float(0x7F800000);
          int am = -1;
          unsigned int negs = 0, par = (s >> r) & 1u;
          for (int k = 0; k < L; ++k) {
            const float v = __fsub_rn(post[P.supp[r][k]], c2v[r][k]);
            const float m = fabsf(v);
            const unsigned int neg = __float_as_uint(v) >> 31;
            negs |= neg << k;
            par ^= neg;
            if (m < n1) {
              n2 = n1;
              n1 = m;
              am = k;
            } else if (m < n2) {
              n2 = m;
            }
          }
          for (int k = 0; k < L; ++k) {
            const float mag = (k == am) ? n2 : n1;
            c2v[r][k] = ((par ^ (negs >> k)) & 1u) ? -mag : mag;
          }
        }
        float U[kMaxDelta * kMaxDelta];
        for (int j = 0; j < nl; ++j) U[j] = 0.0f;
        for (int r = 0; r < P.m_l; ++r)
          for (int k = 0; k < P.supp_len[r]; ++k) U[P.supp[r][k]] = __fadd_rn(U[P.supp[r][k]], c2v[r][k]);
        for (int j = 0; j < nl; ++j) post[j] = __fadd_rn(lam, U[j]);
      }
      unsigned long long e = 0;
      for (int j = 0; j < nl; ++j) e |= (unsigned long long)(post[j] < 0.0f) << j;
      bool ok = true;
      for (int r = 0; r < P.m_l; ++r) ok &= ((unsigned int)(__popcll(e & P.rowmask[r]) & 1) == ((s >> r) & 1u));
      if (ok) {
        conv = true;
        break;
      }
      if (t >= max_iter) break;
    }
    unsigned long long e = 0;
    for (int j = 0; j < nl; ++j) e |= (unsigned long long)(post[j] < 0.0f) << j;
    for (int j = 0; j < nl; ++j) {
      float q = sigmoid_f32(post[j]);
      if (conv && ((e >> j) & 1)) q = fmaxf(q, 0.5f);
      table[(size_t)s * nl + j] = q;
    }
    if (iters) iters[s] = t | (conv ? 0x10000 : 0);
  }
}

// lambda(p) of n probabilities (lead_prior_llr).
__global__ void prior_llr_kernel(const float* __restrict__ p, float* __restrict__ llr, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    llr[i] = llr_f32(__ldg(p + i));
}

template <typename T>
int upload(T** dst, const std::vector<T>& src) {
  if (src.empty()) {
    *dst = nullptr;
    return LEAD_OK;
  }
  if (cudaMalloc(dst, src.size() * sizeof(T)) != cudaSuccess) return LEAD_EOOM;
  LEAD_CUDA_TRY(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return LEAD_OK;
}

#define LEAD_TRY(expr)             \
  do {                             \
    int _rc = (expr);              \
    if (_rc != LEAD_OK) return _rc; \
  } while (0)

int prepare_side(lead_code* code, int s) {
  HostSide& hs = code->side[s];
  DeviceSide& ds = code->dside[s];
  const int nl = code->nl, delta = code->delta;
  std::vector<uint16_t> views(hs.views.begin(), hs.views.end());
  LEAD_TRY(upload(&ds.views, views));
  LEAD_TRY(upload(&ds.partner, hs.partner));
  LEAD_TRY(upload(&ds.qslots, hs.qslots));
  LEAD_TRY(upload(&ds.logicals, hs.logicals));
  LEAD_TRY(upload(&ds.xcls, hs.xcls));
  LEAD_TRY(upload(&ds.cbase, hs.cbase));
  LEAD_TRY(upload(&ds.ckern, hs.ckern));
  // min-sum kernel partner table. One CTA per shot group: thread t = shot sl * order + vertex v,
  // slot (j, t) lives at shared-memory word j * ts + t; entry = partner address | first << 15.
  // Cluster launch: CTA rank r owns vertices r*ts .. r*ts + ts - 1; entry (indexed [j][v]) =
  // partner word address inside its owner | owner rank << 13 | first << 15 (u16, cluster_pa16),
  // or, for larger shapes, address | owner rank << 16 | first << 31 (u32).
  {
    const Geometry g = bp_geometry(code, s);
    const std::vector<uint8_t> pa = partner_table_bytes(code, s, g);
    if (!pa.empty()) {
      uint8_t* d = nullptr;
      LEAD_TRY(upload(&d, pa));
      ds.bp_pa = reinterpret_cast<uint16_t*>(d);
    }
  }
  // syndrome contribution of row pattern x at row a: bit (rB*kRA + rA) = RA[rA][a] * (RB x)[rB]
  std::vector<uint16_t> contrib((size_t)delta << delta, 0);
  for (int a = 0; a < delta; ++a)
    for (int x = 0; x < (1 << delta); ++x) {
      uint32_t c = 0;
      for (int rB = 0; rB < hs.kRB; ++rB) {
        int f = 0;
        for (int b = 0; b < delta; ++b) f ^= ((x >> b) & 1) & hs.RB[rB * delta + b];
        if (!f) continue;
        for (int rA = 0; rA < hs.kRA; ++rA)
          if (hs.RA[rA * delta + a]) c ^= 1u << (rB * hs.kRA + rA);
      }
      contrib[(size_t)a * (1 << delta) + x] = (uint16_t)c;
    }
  uint16_t* dcontrib = nullptr;
  LEAD_TRY(upload(&dcontrib, contrib));
  const int states = 1 << hs.m_l;
  const size_t sz = (size_t)states * (nl + 1);
  if (cudaMalloc(&ds.enumN, sz * sizeof(int32_t)) != cudaSuccess) return LEAD_EOOM;
  if (cudaMalloc(&ds.enumN1, sz * nl * sizeof(int32_t)) != cudaSuccess) return LEAD_EOOM;
  if (cudaMalloc(&ds.ml, states * sizeof(uint64_t)) != cudaSuccess) return LEAD_EOOM;
  unsigned long long* bufs = nullptr;
  // (nl + 1) double-buffered enumeration runs, then the two buffers of the ML recursion
  const size_t nbuf = sz * 2 * (nl + 1) + (size_t)states * 2;
  if (cudaMalloc(&bufs, nbuf * sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(dcontrib);
    return LEAD_EOOM;
  }
  enumerate_kernel<<<nl + 1, 512>>>(delta, hs.m_l, dcontrib, bufs, ds.enumN, ds.enumN1);
  cudaError_t e1 = cudaGetLastError();
  ml_kernel<<<1, 512>>>(delta, hs.m_l, dcontrib, bufs + sz * 2 * (nl + 1), ds.ml);
  cudaError_t e2 = cudaGetLastError();
  cudaError_t e3 = cudaDeviceSynchronize();
  cudaFree(bufs);
  cudaFree(dcontrib);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return LEAD_ECUDA;
  return LEAD_OK;
}

}  // namespace

int prepare_device(lead_code* code, int device) {
  if (code->device == device) return LEAD_OK;
  if (code->device >= 0) return LEAD_ESTATE;
  int rc = jit_compile(code, nullptr);       // host-only; skipped if lead_code_compile ran
  if (rc != LEAD_OK) return rc;
  LEAD_CUDA_TRY(cudaSetDevice(device));
  LEAD_CUDA_TRY(cudaFree(nullptr));           // make the device's primary context current
  code->device = device;
  for (int s = 0; s < 2; ++s) {
    rc = prepare_side(code, s);
    if (rc != LEAD_OK) {
      release_device(code);
      return rc;
    }
  }
  if (cudaMalloc(&code->d_check, 5 * sizeof(unsigned long long)) != cudaSuccess) {
    release_device(code);
    return LEAD_EOOM;
  }
  if (cudaMemset(code->d_check, 0, 5 * sizeof(unsigned long long)) != cudaSuccess) {
    release_device(code);
    return LEAD_ECUDA;
  }
  rc = jit_load(code);
  if (rc != LEAD_OK) {
    release_device(code);
    return rc;
  }
  return LEAD_OK;
}

void release_device(lead_code* code) {
  if (code->device < 0) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(code->device);
  jit_unload(code);
  for (auto& ds : code->dside) {
    cudaFree(ds.views);
    cudaFree(ds.partner);
    cudaFree(ds.qslots);
    cudaFree(ds.enumN);
    cudaFree(ds.enumN1);
    cudaFree(ds.ml);
    cudaFree(ds.logicals);
    cudaFree(ds.bp_pa);
    cudaFree(ds.xcls);
    cudaFree(ds.cbase);
    cudaFree(ds.ckern);
    ds = DeviceSide{};
  }
  cudaFree(code->d_check);
  code->d_check = nullptr;
  if (prev >= 0) cudaSetDevice(prev);
  code->device = -1;
}

int check_device(const lead_code* code) {
  if (!code) return LEAD_EINVAL;
  if (code->device < 0) return LEAD_ESTATE;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return LEAD_ECUDA;
  return cur == code->device ? LEAD_OK : LEAD_ESTATE;
}

int launch_table(const lead_code* code, int side, double p, float* table, cudaStream_t stream, int estimator,
                 int32_t* iters) {
  if (!(p > 0.0 && p < 0.5)) return LEAD_EINVAL;
  const HostSide& hs = code->side[side];
  const DeviceSide& ds = code->dside[side];
  if (estimator == LEAD_EST_MINSUM) {
    // the local code length Delta^2 bounds the iterations (the paper runs BP up to the length)
    const int S = 1 << hs.m_l;
    minsum_table_kernel<<<(S + 127) / 128, 128, 0, stream>>>(hs.params, code->nl, (float)p, code->nl, table,
                                                              iters);
    LEAD_CUDA_TRY(cudaGetLastError());
    return LEAD_OK;
  }
  if (estimator != LEAD_EST_EXACT) return LEAD_EINVAL;
  const double r = p / (1.0 - p);
  const int total = (1 << hs.m_l) * code->nl;
  const int threads = 256;
  const int blocks = (total + threads - 1) / threads;
  table_kernel<<<blocks, threads, 0, stream>>>(code->nl, hs.m_l, r, ds.enumN, ds.enumN1, ds.ml, table);
  LEAD_CUDA_TRY(cudaGetLastError());
  return LEAD_OK;
}

int check_result(const lead_code* code, void* stream) {
#if LEAD_CHECKED
  // a call being captured into a CUDA graph cannot wait: its record is read by the next call
  // that runs eagerly
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  LEAD_CUDA_TRY(cudaStreamIsCapturing((cudaStream_t)stream, &cap));
  if (cap != cudaStreamCaptureStatusNone) return LEAD_OK;
  unsigned long long rec[4];
  LEAD_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  LEAD_CUDA_TRY(cudaMemcpy(rec, code->d_check, sizeof(rec), cudaMemcpyDeviceToHost));
  if (rec[0] == 0) return LEAD_OK;
  std::memcpy(code->last_check, rec, sizeof(rec));
  LEAD_CUDA_TRY(cudaMemset(code->d_check, 0, sizeof(rec)));
  return LEAD_ECHECK;
#else
  (void)code;
  (void)stream;
  return LEAD_OK;
#endif
}

}  // namespace lead

extern "C" {

int lead_build_flags(void) { return LEAD_CHECKED ? LEAD_BUILD_CHECKED : 0; }

int lead_code_check_record(const lead_code* code, uint64_t record[4]) {
  if (!code || !record) return LEAD_EINVAL;
  for (int i = 0; i < 4; ++i) record[i] = code->last_check[i];
  return LEAD_OK;
}

int lead_code_device_errors(const lead_code* code, uint32_t* flags, int32_t clear) {
  if (!code || !flags) return LEAD_EINVAL;
  if (code->device < 0) return LEAD_ESTATE;
  int cur = -1;
  LEAD_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != code->device) return LEAD_ESTATE;
  unsigned long long w = 0;
  LEAD_CUDA_TRY(cudaMemcpy(&w, code->d_check + 4, sizeof(w), cudaMemcpyDeviceToHost));
  *flags = (uint32_t)w;
  if (clear) LEAD_CUDA_TRY(cudaMemset(code->d_check + 4, 0, sizeof(w)));
  return LEAD_OK;
}

int lead_code_prepare(lead_code* code, int32_t device) {
  if (!code || device < 0) return LEAD_EINVAL;
  return lead::prepare_device(code, device);
}

int lead_code_get_enumerators(const lead_code* code, int32_t side, int32_t* N, int32_t* N1,
                              uint64_t* ml) {
  if (!code || side < 0 || side > 1) return LEAD_EINVAL;
  if (code->device < 0) return LEAD_ESTATE;
  const auto& hs = code->side[side];
  const auto& ds = code->dside[side];
  const size_t sz = (size_t)(1 << hs.m_l) * (code->nl + 1);
  if (N) LEAD_CUDA_TRY(cudaMemcpy(N, ds.enumN, sz * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (N1) LEAD_CUDA_TRY(cudaMemcpy(N1, ds.enumN1, sz * code->nl * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (ml) LEAD_CUDA_TRY(cudaMemcpy(ml, ds.ml, (size_t)(1 << hs.m_l) * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  return LEAD_OK;
}

int lead_prior_llr(const float* p, float* llr, int64_t n, void* stream) {
  if (n < 0) return LEAD_EINVAL;
  if (n == 0) return LEAD_OK;
  if (!p || !llr) return LEAD_EINVAL;
  int dev = 0;
  LEAD_CUDA_TRY(cudaGetDevice(&dev));
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)lead::sm_count(dev) * 8);
  lead::prior_llr_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(p, llr, n);
  LEAD_CUDA_TRY(cudaGetLastError());
  return LEAD_OK;
}

int lead_local_table(const lead_code* code, int32_t side, double p, float* table, void* stream) {
  if (!code || !table || side < 0 || side > 1) return LEAD_EINVAL;
  int rc = lead::check_device(code);
  if (rc != LEAD_OK) return rc;
  return lead::launch_table(code, side, p, table, (cudaStream_t)stream, LEAD_EST_EXACT, nullptr);
}

int lead_local_table_est(const lead_code* code, int32_t side, double p, int32_t estimator, float* table,
                         int32_t* iters, void* stream) {
  if (!code || !table || side < 0 || side > 1) return LEAD_EINVAL;
  if (estimator != LEAD_EST_EXACT && estimator != LEAD_EST_MINSUM) return LEAD_EINVAL;
  int rc = lead::check_device(code);
  if (rc != LEAD_OK) return rc;
  if (iters && estimator == LEAD_EST_EXACT) {       // the exact estimator is one-shot: 1, converged
    const int S = 1 << code->side[side].m_l;
    lead::fill_i32_kernel<<<(S + 255) / 256, 256, 0, (cudaStream_t)stream>>>(iters, S, 1 | 0x10000);
    LEAD_CUDA_TRY(cudaGetLastError());
  }
  return lead::launch_table(code, side, p, table, (cudaStream_t)stream, estimator, iters);
}

}  // extern "C"
