// Noise sampling (Sec. IV-A) and syndromes s_Z = H_Z e_X, s_X = H_X e_Z, and the residual /
// logical check of a correction.
#include <cuda_runtime.h>

#include <algorithm>

#include "lead_device.cuh"

namespace lead {
int check_device(const lead_code* code);

namespace {

struct SampleArgs {
  int32_t n, words_n, order, nl, noise, spb;
  uint32_t tb, t1, t2, t3;
  uint32_t k0, k1;
  uint64_t offset;
  int64_t shots;
  uint32_t* err_x;
  uint32_t* err_z;
  uint32_t* syn_z;
  uint32_t* syn_x;
  const uint16_t* views0;
  const uint16_t* views1;
};

// The local syndrome of vertex v: gather the view's bits of a packed error row held in shared
// memory and take the parity of each local check row.
__device__ __forceinline__ uint32_t local_syndrome(const uint32_t* e, const uint16_t* __restrict__ views,
                                                   int v, const SideParams& P) {
  uint64_t x = 0;
  for (int j = 0; j < P.nl; ++j) {
    const int q = __ldg(views + v * P.nl + j);
    x |= (uint64_t)((e[q >> 5] >> (q & 31)) & 1u) << j;
  }
  uint32_t s = 0;
  for (int r = 0; r < P.m_l; ++r) s |= (uint32_t)(__popcll(x & P.rowmask[r]) & 1) << r;
  return s;
}

__device__ __forceinline__ void or_field(uint32_t* row, int pos, int len, uint32_t val) {
  if (!val) return;
  const int w = pos >> 5, sh = pos & 31;
  atomicOr(row + w, val << sh);
  if (sh + len > 32) atomicOr(row + w + 1, val >> (32 - sh));
}

__global__ void sample_kernel(SampleArgs a, __grid_constant__ const SideParams P0,
                              __grid_constant__ const SideParams P1) {
  extern __shared__ uint32_t smem[];
  const int spb = a.spb;
  uint32_t* ex = smem;
  uint32_t* ez = ex + spb * a.words_n;
  uint32_t* sz = ez + spb * a.words_n;
  uint32_t* sx = sz + spb * P0.words_m;
  const int total = spb * (2 * a.words_n + P0.words_m + P1.words_m);
  const int groups = (a.n + 3) >> 2;
  const bool want_x = a.err_x || a.syn_z;
  const bool want_z = a.err_z || a.syn_x;
  for (int64_t base = (int64_t)blockIdx.x * spb; base < a.shots; base += (int64_t)gridDim.x * spb) {
    const int nsh = (int)rows_left(spb, a.shots - base);
    for (int i = threadIdx.x; i < total; i += blockDim.x) smem[i] = 0u;
    __syncthreads();
    for (int idx = threadIdx.x; idx < nsh * groups; idx += blockDim.x) {
      const int sl = idx / groups, g = idx - sl * groups;
      const uint64_t shot = a.offset + (uint64_t)(base + sl);
      const uint4 u = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)shot, (uint32_t)(shot >> 32), 0u),
                                    a.k0, a.k1);
      const uint32_t us[4] = {u.x, u.y, u.z, u.w};
      uint32_t nx = 0, nz = 0;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        if (4 * g + l >= a.n) break;
        uint32_t x, z;
        if (a.noise == LEAD_NOISE_DEPOL) {
          x = us[l] < a.t2;
          z = (us[l] >= a.t1) & (us[l] < a.t3);
        } else {
          const uint32_t f = us[l] < a.tb;
          x = (a.noise == LEAD_NOISE_X) ? f : 0u;
          z = (a.noise == LEAD_NOISE_Z) ? f : 0u;
        }
        nx |= x << l;
        nz |= z << l;
      }
      const int i0 = 4 * g;
      if (nx) atomicOr(ex + sl * a.words_n + (i0 >> 5), nx << (i0 & 31));
      if (nz) atomicOr(ez + sl * a.words_n + (i0 >> 5), nz << (i0 & 31));
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nsh * a.order; idx += blockDim.x) {
      const int sl = idx / a.order, v = idx - sl * a.order;
      if (a.syn_z && want_x)
        or_field(sz + sl * P0.words_m, v * P0.m_l, P0.m_l,
                 local_syndrome(ex + sl * a.words_n, a.views0, v, P0));
      if (a.syn_x && want_z)
        or_field(sx + sl * P1.words_m, v * P1.m_l, P1.m_l,
                 local_syndrome(ez + sl * a.words_n, a.views1, v, P1));
    }
    __syncthreads();
    const int64_t r0 = base;
    for (int i = threadIdx.x; i < nsh * a.words_n; i += blockDim.x) {
      if (a.err_x) a.err_x[r0 * a.words_n + i] = ex[i];
      if (a.err_z) a.err_z[r0 * a.words_n + i] = ez[i];
    }
    if (a.syn_z)
      for (int i = threadIdx.x; i < nsh * P0.words_m; i += blockDim.x) a.syn_z[r0 * P0.words_m + i] = sz[i];
    if (a.syn_x)
      for (int i = threadIdx.x; i < nsh * P1.words_m; i += blockDim.x) a.syn_x[r0 * P1.words_m + i] = sx[i];
    __syncthreads();
  }
}

struct CheckArgs {
  int32_t words_n, order, nl, k, spb;
  int64_t shots;
  const uint32_t* err;
  const uint32_t* corr;
  const uint16_t* views;
  const uint32_t* logicals;
  uint8_t* fail;
};

// Residual r = err + corr: bit 0 of fail = some local check of r is violated (H r != 0);
// bit 1 = H r = 0 and some logical operator of the other type has odd overlap with r.
__global__ void check_kernel(CheckArgs a, __grid_constant__ const SideParams P) {
  extern __shared__ uint32_t smem[];
  const int spb = a.spb;
  uint32_t* r = smem;
  int* flags = (int*)(r + spb * a.words_n);
  for (int64_t base = (int64_t)blockIdx.x * spb; base < a.shots; base += (int64_t)gridDim.x * spb) {
    const int nsh = (int)rows_left(spb, a.shots - base);
    for (int i = threadIdx.x; i < nsh * a.words_n; i += blockDim.x)
      r[i] = a.err[base * a.words_n + i] ^ a.corr[base * a.words_n + i];
    for (int i = threadIdx.x; i < 2 * spb; i += blockDim.x) flags[i] = 0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < nsh * a.order; idx += blockDim.x) {
      const int sl = idx / a.order, v = idx - sl * a.order;
      if (local_syndrome(r + sl * a.words_n, a.views, v, P)) atomicOr(flags + 2 * sl, 1);
    }
    for (int idx = threadIdx.x; idx < nsh * a.k; idx += blockDim.x) {
      const int sl = idx / a.k, l = idx - sl * a.k;
      uint32_t par = 0;
      for (int w = 0; w < a.words_n; ++w) par ^= __popc(r[sl * a.words_n + w] & __ldg(a.logicals + l * a.words_n + w));
      if (par & 1) atomicOr(flags + 2 * sl + 1, 1);
    }
    __syncthreads();
    for (int sl = threadIdx.x; sl < nsh; sl += blockDim.x) {
      const int bad = flags[2 * sl];
      a.fail[base + sl] = (uint8_t)(bad ? 1 : (flags[2 * sl + 1] ? 2 : 0));
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace lead

extern "C" {

int lead_sample(const lead_code* code, int32_t noise, double p, int64_t shots, uint64_t seed,
                uint64_t shot_offset, uint32_t* err_x, uint32_t* err_z, uint32_t* syn_z,
                uint32_t* syn_x, void* stream) {
  using namespace lead;
  int rc = check_device(code);
  if (rc != LEAD_OK) return rc;
  if (shots < 0 || !(p >= 0.0 && p < 1.0)) return LEAD_EINVAL;
  if (noise != LEAD_NOISE_X && noise != LEAD_NOISE_Z && noise != LEAD_NOISE_DEPOL) return LEAD_EINVAL;
  if (shots == 0) return LEAD_OK;
  SampleArgs a{};
  a.n = code->n;
  a.words_n = code->words_n;
  a.order = code->order;
  a.nl = code->nl;
  a.noise = noise;
  const double two32 = 4294967296.0;
  auto thr = [&](double x) -> uint32_t {
    double t = x * two32;
    return t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;   // floor for 0 <= t < 2^32
  };
  a.tb = thr(p);
  a.t1 = thr(p / 3.0);
  a.t2 = thr((2.0 * p) / 3.0);
  a.t3 = thr(p);
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  a.offset = shot_offset;
  a.shots = shots;
  a.err_x = err_x;
  a.err_z = err_z;
  a.syn_z = syn_z;
  a.syn_x = syn_x;
  a.views0 = code->dside[0].views;
  a.views1 = code->dside[1].views;
  const SideParams& P0 = code->side[0].params;
  const SideParams& P1 = code->side[1].params;
  const int groups = (code->n + 3) / 4;
  a.spb = groups >= 512 ? 1 : (512 + groups - 1) / groups;
  const size_t smem = (size_t)a.spb * (2 * a.words_n + P0.words_m + P1.words_m) * sizeof(uint32_t);
  if (smem > 48 * 1024) return LEAD_EINVAL;
  const int64_t batches = (shots + a.spb - 1) / a.spb;
  const int64_t blocks = std::min<int64_t>(batches, (int64_t)sm_count(code->device) * 8);
  sample_kernel<<<(unsigned)blocks, 256, smem, (cudaStream_t)stream>>>(a, P0, P1);
  LEAD_CUDA_TRY(cudaGetLastError());
  return LEAD_OK;
}

int lead_check(const lead_code* code, int32_t side, const uint32_t* err, const uint32_t* corr,
               int64_t shots, uint8_t* fail, void* stream) {
  using namespace lead;
  int rc = check_device(code);
  if (rc != LEAD_OK) return rc;
  if (side < 0 || side > 1 || shots < 0) return LEAD_EINVAL;
  if (shots == 0) return LEAD_OK;          // empty batch: nothing to read or write
  if (!err || !corr || !fail) return LEAD_EINVAL;
  CheckArgs a{};
  a.words_n = code->words_n;
  a.order = code->order;
  a.nl = code->nl;
  a.k = code->k;
  a.shots = shots;
  a.err = err;
  a.corr = corr;
  a.views = code->dside[side].views;
  a.logicals = code->dside[side].logicals;
  a.fail = fail;
  a.spb = code->order >= 256 ? 1 : 256 / code->order;
  const size_t smem = (size_t)a.spb * a.words_n * sizeof(uint32_t) + 2 * a.spb * sizeof(int);
  if (smem > 48 * 1024) return LEAD_EINVAL;
  const int64_t batches = (shots + a.spb - 1) / a.spb;
  const int64_t blocks = std::min<int64_t>(batches, (int64_t)sm_count(code->device) * 8);
  check_kernel<<<(unsigned)blocks, 256, smem, (cudaStream_t)stream>>>(a, code->side[side].params);
  LEAD_CUDA_TRY(cudaGetLastError());
  return LEAD_OK;
}

}  // extern "C"
