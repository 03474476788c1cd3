// Run-time specialisation of the min-sum kernel to a code side (NVRTC -> cubin for sm_103a),
// loaded and launched through the CUDA runtime's library-management API.
//
// The kernel source (bp_jit_kernel.cuh with bp_jit_args.h and lead_math.cuh) is compiled into
// the library as text. For each side the host prepends a prelude with the side's sizes and the
// supports of its local check rows, so every edge loop of the kernel has compile-time trip
// counts and shared-memory offsets.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "bp_jit_args.h"
#include "lead_internal.h"
#include "lead_jit_source.inc"   // generated at build time: kLeadJitSource

namespace lead {

namespace {

}  // namespace

// Bytes of one stored LLR in a precision mode.
static size_t msg_bytes(int prec) { return prec == LEAD_PREC_FP32 ? 4 : 2; }

Geometry bp_geometry(const lead_code* code, int side, int prec, int spb_req, int cluster_req) {
  const SideParams& P = code->side[side].params;
  Geometry g{};
  // With one shot per CTA (or per cluster) the staged syndrome row lives in the posterior array
  // (which the first iteration writes only after the prologue has read the syndromes) and the
  // correction bits in the prior array (dead once the shot has stopped); only the cluster
  // kernel's two verdict words follow the messages.
  // (the posterior and prior arrays start at multiples of one array's bytes, which must keep
  // the 4-byte alignment of the words stored there)
  auto aliased = [&](int ts, int spb, size_t mb) {
    const size_t region = (size_t)ts * code->nl * mb;     // one of the three message arrays
    return spb == 1 && region % 4 == 0 && region >= sizeof(uint32_t) * std::max<size_t>(P.words_m, code->words_n);
  };
  auto smem_for = [&](int ts, int spb, size_t mb) {
    const size_t msgs = ((size_t)ts * code->nl * 3 * mb + 15) & ~size_t(15);
    if (aliased(ts, spb, mb)) return msgs + 16;
    // staged syndromes, correction bits and three verdict words per shot (one spare word)
    return msgs + sizeof(uint32_t) * ((size_t)spb * P.words_m + (size_t)spb * code->words_n + 3 * (size_t)spb + 1);
  };
  // The split of shots and vertices over CTAs is fixed by the binary32 footprint, so every
  // precision mode shares one partner table; the 16-bit modes only need less shared memory.
  g.spb = bp_shots_per_block(code);
  g.cluster = 1;
  g.ts = g.spb * code->order;
  size_t smem32 = smem_for(g.ts, g.spb, 4);
  // a shot whose state does not leave room for two CTAs per SM is split over a thread-block
  // cluster (distributed shared memory), 2, 4 or 8 CTAs
  while (smem32 > 120u * 1024u && g.cluster < 8) {
    g.cluster *= 2;
    g.spb = 1;
    g.ts = (code->order + g.cluster - 1) / g.cluster;
    smem32 = smem_for(g.ts, 1, 4);
  }
  if (spb_req > 0 && g.cluster == 1) {     // another number of shots per CTA (autotuning)
    g.spb = spb_req;
    g.ts = g.spb * code->order;
  }
  if (cluster_req >= 1 && g.cluster > 1) {  // another cluster size, or one CTA per shot (autotuning)
    g.cluster = cluster_req;
    g.spb = 1;
    g.ts = (code->order + g.cluster - 1) / g.cluster;
  }
  g.smem = smem_for(g.ts, g.spb, msg_bytes(prec));
  g.alias = aliased(g.ts, g.spb, msg_bytes(prec));
  g.block = (g.ts + 31) / 32 * 32;
  // CTAs per SM that shared memory allows (227 KB usable, 1 KB reserved per CTA), capped so
  // that each thread keeps at least 48 registers (compile_one steps down while the register cap
  // this implies makes the compiler spill)
  int by_smem = (int)((227u * 1024u) / (g.smem + 1024));
  int by_regs = 65536 / (g.block * 48);
  g.minblocks = std::max(1, std::min(by_smem, by_regs));
  return g;
}

namespace {

std::string prelude(const lead_code* code, int side, const Geometry& g, int prec) {
  const SideParams& P = code->side[side].params;
  int kmax = 1;
  for (int r = 0; r < P.m_l; ++r) kmax = std::max(kmax, P.supp_len[r]);
  std::ostringstream s;
#if defined(LEAD_CHECKED) && LEAD_CHECKED
  s << "#define LEAD_CHECKED 1\n";       // the checked build's kernels test their table indices
#endif
  s << "#define LEAD_NL " << code->nl << "\n"
    << "#define LEAD_ML " << P.m_l << "\n"
    << "#define LEAD_TS " << g.ts << "\n"
    << "#define LEAD_BLOCK " << g.block << "\n"
    << "#define LEAD_MINBLOCKS " << g.minblocks << "\n"
    << "#define LEAD_KMAX " << kmax << "\n"
    << "#define LEAD_SPB " << g.spb << "\n"
    << "#define LEAD_CLUSTER " << g.cluster << "\n"
    << "#define LEAD_PREC " << prec << "\n"
    << "#define LEAD_PA16 " << (cluster_pa16(g, code->nl) ? 1 : 0) << "\n"
    << "#define LEAD_ALIAS " << (g.alias ? 1 : 0) << "\n";
  // the local rows touching every slot j (increasing) and j's position in each row's support
  std::vector<std::vector<std::pair<int, int>>> rows_of(code->nl);
  for (int r = 0; r < P.m_l; ++r)
    for (int k = 0; k < P.supp_len[r]; ++k) rows_of[P.supp[r][k]].push_back({r, k});
  int jmax = 1;
  for (const auto& v : rows_of) jmax = std::max(jmax, (int)v.size());
  s << "#define LEAD_JMAX " << jmax << "\n"
    << "namespace lead_jit {\n";
  s << "__device__ constexpr int kLen[" << P.m_l << "] = {";
  for (int r = 0; r < P.m_l; ++r) s << (r ? "," : "") << P.supp_len[r];
  s << "};\n__device__ constexpr int kSupp[" << P.m_l << "][" << kmax << "] = {";
  for (int r = 0; r < P.m_l; ++r) {
    s << (r ? ",{" : "{");
    for (int k = 0; k < kmax; ++k) s << (k ? "," : "") << (k < P.supp_len[r] ? (int)P.supp[r][k] : 0);
    s << "}";
  }
  s << "};\n__device__ constexpr int kJLen[" << code->nl << "] = {";
  for (int j = 0; j < code->nl; ++j) s << (j ? "," : "") << rows_of[j].size();
  for (int part = 0; part < 2; ++part) {
    s << "};\n__device__ constexpr int " << (part ? "kJPos" : "kJRow") << "[" << code->nl << "][" << jmax << "] = {";
    for (int j = 0; j < code->nl; ++j) {
      s << (j ? ",{" : "{");
      for (int i = 0; i < jmax; ++i) {
        const int val = i < (int)rows_of[j].size() ? (part ? rows_of[j][i].second : rows_of[j][i].first) : 0;
        s << (i ? "," : "") << val;
      }
      s << "}";
    }
  }
  // the local rows over the two words of the kernel's hard-decision bits: local index j < 32 at
  // bit nlo - 1 - j of the low word (nlo = min(nl, 32)), j >= 32 at bit nl - 1 - j of the high one
  const int nlo = std::min(code->nl, 32);
  for (int part = 0; part < 2; ++part) {
    s << "};\n__device__ constexpr unsigned int " << (part ? "kRowHi" : "kRowLo") << "[" << P.m_l << "] = {";
    for (int r = 0; r < P.m_l; ++r) {
      unsigned int w = 0;
      for (int j = 0; j < code->nl; ++j) {
        if (!((P.rowmask[r] >> j) & 1ull)) continue;
        if (part == 0 && j < 32) w |= 1u << (nlo - 1 - j);
        if (part == 1 && j >= 32) w |= 1u << (code->nl - 1 - j);
      }
      s << (r ? "," : "") << w << "u";
    }
  }
  s << "};\n}\n";
  return s.str();
}

}  // namespace

// NVRTC compile of the kernel for one side and precision mode into hs.bp_cubin[prec].
namespace {

// Sum of the "N bytes spill stores" figures in a ptxas -v report.
long spill_bytes(const std::string& log) {
  long total = 0;
  const std::string key = " bytes spill stores";
  for (size_t pos = log.find(key); pos != std::string::npos; pos = log.find(key, pos + 1)) {
    size_t b = pos;
    while (b > 0 && log[b - 1] >= '0' && log[b - 1] <= '9') --b;
    if (b < pos) total += std::strtol(log.c_str() + b, nullptr, 10);
  }
  return total;
}

// One NVRTC compile; returns the cubin (empty on failure) and the compiler log.
int nvrtc_build(const std::string& src, int maxreg, std::vector<char>* cubin, std::string* log) {
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "lead_bp_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
    return LEAD_ECUDA;
  const std::string regopt = "--maxrregcount=" + std::to_string(maxreg);
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=false", "-lineinfo",
                        regopt.c_str(), "--ptxas-options=-v"};
  const nvrtcResult rc = nvrtcCompileProgram(prog, 6, opts);
  size_t logn = 0;
  nvrtcGetProgramLogSize(prog, &logn);
  log->assign(logn, '\0');
  if (logn) nvrtcGetProgramLog(prog, &(*log)[0]);
  log->resize(std::strlen(log->c_str()));          // the reported size counts the terminating NUL
  if (rc != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    return LEAD_ECUDA;
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  cubin->resize(n);
  nvrtcGetCUBIN(prog, cubin->data());
  nvrtcDestroyProgram(&prog);
  return LEAD_OK;
}

}  // namespace

// Spill stores tolerated at a register cap: a few words, which stay in L1.
constexpr long kSpillSlack = 16;

// NVRTC compile of the kernel for one side and precision mode into hs.bp_cubin[prec]. The
// resident CTAs per SM start at what shared memory allows and step down while the register
// cap that occupancy implies makes the compiler spill more than kSpillSlack bytes.
int compile_one(lead_code* code, int side, int prec, std::string* log_out) {
  HostSide& hs = code->side[side];
  if (!hs.bp_cubin[prec].empty()) return LEAD_OK;
  Geometry g = bp_geometry(code, side, prec);
  if (g.block > 1024 || (size_t)code->nl * g.ts >= 32768 || g.smem > 227u * 1024u) return LEAD_EINVAL;
  // LEAD_JIT_PTXAS_VERBOSE=1 keeps the assembler's register / spill report in the log
  const char* verbose = std::getenv("LEAD_JIT_PTXAS_VERBOSE");
  std::vector<char> cubin;
  std::string log;
  int maxreg = 0;
  std::ostringstream tries;
  for (;; --g.minblocks) {
    // registers per thread that let LEAD_MINBLOCKS CTAs of this size share an SM
    maxreg = std::min(255, (65536 / (g.block * g.minblocks)) & ~7);
    const std::string src = prelude(code, side, g, prec) + kLeadJitSource;
    const int rc = nvrtc_build(src, maxreg, &cubin, &log);
    if (rc != LEAD_OK) {
      if (log_out) *log_out += log;
      return rc;
    }
    const long spill = spill_bytes(log);
    tries << "  " << g.minblocks << " CTA(s) per SM, <= " << maxreg << " registers: " << spill << " B spilled\n";
    if (g.minblocks == 1 || spill <= kSpillSlack) break;
  }
  if (log_out) {
    std::ostringstream gs;
    gs << "side " << side << " precision " << prec << ": " << (g.cluster > 1 ? "cluster of " : "") << g.cluster
       << " CTA(s) x " << g.block << " threads, " << g.ts << " slots per CTA row, " << g.spb
       << " shot(s) per CTA, " << g.smem << " B shared memory, " << g.minblocks << " CTA(s) per SM, <= " << maxreg
       << " registers\n";
    *log_out += gs.str() + tries.str();
    if (verbose && verbose[0] == '1') *log_out += log;
  }
  hs.bp_cubin[prec] = std::move(cubin);
  hs.bp_block = g.block;
  hs.bp_spb = g.spb;
  hs.bp_cluster = g.cluster;
  hs.bp_smem[prec] = g.smem;
  hs.bp_maxreg[prec] = maxreg;
  return LEAD_OK;
}

namespace {

// Loads the compiled kernel of (side, prec) on the current device.
int load_one(lead_code* code, int side, int prec) {
  HostSide& hs = code->side[side];
  DeviceSide& ds = code->dside[side];
  if (ds.bp_func[prec]) return LEAD_OK;
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
  if (cudaLibraryLoadData(&lib, hs.bp_cubin[prec].data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess)
    return LEAD_ECUDA;
  int per_sm = 0;
  const char* name = hs.bp_cluster > 1 ? "lead_bp_jit_cluster" : "lead_bp_jit";
  if (cudaLibraryGetKernel(&kern, lib, name) != cudaSuccess ||
      cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs.bp_smem[prec]) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)kern, hs.bp_block, hs.bp_smem[prec]) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaLibraryUnload(lib);
    return LEAD_ECUDA;
  }
  ds.bp_module[prec] = lib;
  ds.bp_func[prec] = kern;
  ds.bp_per_sm[prec] = per_sm;
  return LEAD_OK;
}

}  // namespace

int jit_compile(lead_code* code, std::string* log_out) {
  for (int side = 0; side < 2; ++side) {
    const int rc = compile_one(code, side, LEAD_PREC_FP32, log_out);
    if (rc != LEAD_OK) return rc;
  }
  return LEAD_OK;
}

int jit_load(lead_code* code) {
  for (int side = 0; side < 2; ++side) {
    const int rc = load_one(code, side, LEAD_PREC_FP32);
    if (rc != LEAD_OK) return rc;
  }
  return LEAD_OK;
}

int jit_ensure(const lead_code* ccode, int side, int prec) {
  lead_code* code = const_cast<lead_code*>(ccode);   // the kernel cache is not part of the code's value
  if (prec < 0 || prec >= kPrecModes) return LEAD_EINVAL;
  std::lock_guard<std::mutex> lock(code->jit_mu);
  int rc = compile_one(code, side, prec, nullptr);
  if (rc != LEAD_OK) return rc;
  return load_one(code, side, prec);
}

void release_tuned(TunedKernel& t) {
  if (t.owned && t.lib) cudaLibraryUnload(static_cast<cudaLibrary_t>(t.lib));
  cudaFree(t.pa);
  t = TunedKernel{};
}

void jit_unload(lead_code* code) {
  for (auto& ds : code->dside)
    for (int prec = 0; prec < kPrecModes; ++prec) {
      for (auto& t : ds.tuned[prec]) release_tuned(t);
      ds.tuned[prec].clear();
      if (ds.bp_module[prec]) cudaLibraryUnload(static_cast<cudaLibrary_t>(ds.bp_module[prec]));
      ds.bp_module[prec] = nullptr;
      ds.bp_func[prec] = nullptr;
    }
}

// The tuned launch shape for prior p: the one whose tuning prior is nearest on a log scale, or
// null (the default kernel) when none was tuned.
const TunedKernel* tuned_for(const DeviceSide& ds, int prec, double p) {
  const TunedKernel* best = nullptr;
  double dbest = 0.0;
  for (const TunedKernel& t : ds.tuned[prec]) {
    const double d = std::fabs(std::log(std::max(p, 1e-12) / t.p));
    if (!best || d < dbest) {
      best = &t;
      dbest = d;
    }
  }
  return best;
}

int jit_launch_bp(const lead_code* code, int side, int prec, const BPJitArgs& args, int sm_count, void* stream) {
  const HostSide& hs = code->side[side];
  const DeviceSide& ds = code->dside[side];
  if (prec < 0 || prec >= kPrecModes) return LEAD_EINVAL;
  if (prec != LEAD_PREC_FP32) {          // loaded on first use, under the code's lock
    const int rc = jit_ensure(code, side, prec);
    if (rc != LEAD_OK) return rc;
  } else if (!ds.bp_func[prec]) {
    return LEAD_ESTATE;
  }
  const TunedKernel* t = tuned_for(ds, prec, args.p);
  const int spb = t ? t->spb : hs.bp_spb, cl = t ? t->cluster : hs.bp_cluster;
  const int per_sm = t ? t->per_sm : ds.bp_per_sm[prec], block = t ? t->block : hs.bp_block;
  const size_t smem = t ? t->smem : hs.bp_smem[prec];
  const long long groups = (args.shots + spb - 1) / spb;     // shots per CTA or per cluster
  const long long units = std::max<long long>(1, ((long long)sm_count * per_sm) / cl);
  const long long blocks = std::min<long long>(groups, units) * cl;
  BPJitArgs a = args;
  a.spb = spb;
  if (t && t->pa) a.pa = t->pa;        // the partner table of the tuned shape
  void* params[] = {&a};
  if (cudaLaunchKernel(t ? t->func : ds.bp_func[prec], dim3((unsigned)blocks), dim3(block), params, smem,
                       static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LEAD_ECUDA;
  return LEAD_OK;
}

// Autotuning of one side's kernel in one precision mode over its launch shape: the shots per CTA
// (one-CTA codes: one to four times the default, where the block and shared memory allow) or
// the cluster size (codes split over a cluster: 2, 3, 4 or 7 CTAs, or one CTA per shot where a
// 16-bit mode's state fits) and, for each, the resident
// CTAs per SM (the register cap per thread) from what shared memory allows down to two fewer.
// Every candidate is compiled, loaded and timed (CUDA events, one warm-up and two timed calls of
// lead_decode) on `shots` shots sampled at p, and the fastest is kept as the shape of later calls
// whose prior is nearest to p on a log scale (how many iterations shots take, and how unevenly,
// decides which shape wins). Every candidate runs the same arithmetic on every shot, so the
// outputs do not depend on the choice.
int autotune_one(lead_code* code, int side, int prec, double p, int64_t shots, std::string* report) {
  HostSide& hs = code->side[side];
  DeviceSide& ds = code->dside[side];
  int rc = jit_ensure(code, side, prec);            // the default kernel, compiled and loaded
  if (rc != LEAD_OK) return rc;
  const int wm = hs.params.words_m, wn = code->words_n;
  uint32_t *err = nullptr, *syn = nullptr, *corr = nullptr;
  uint8_t* st = nullptr;
  void* ws = nullptr;
  const size_t wsb = decode_workspace_bytes(code, side);
  cudaStream_t stream = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    cudaFree(err);
    cudaFree(syn);
    cudaFree(corr);
    cudaFree(st);
    cudaFree(ws);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (stream) cudaStreamDestroy(stream);
  };
  if (cudaMalloc(&err, sizeof(uint32_t) * shots * wn) != cudaSuccess ||
      cudaMalloc(&syn, sizeof(uint32_t) * shots * wm) != cudaSuccess ||
      cudaMalloc(&corr, sizeof(uint32_t) * shots * wn) != cudaSuccess || cudaMalloc(&st, shots) != cudaSuccess ||
      cudaMalloc(&ws, wsb) != cudaSuccess) {
    cleanup();
    return LEAD_EOOM;
  }
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cleanup();
    return LEAD_ECUDA;
  }
  rc = lead_sample(code, side == 0 ? LEAD_NOISE_X : LEAD_NOISE_Z, p, shots, 0x5EEDull, 0, side == 0 ? err : nullptr,
                   side == 0 ? nullptr : err, side == 0 ? syn : nullptr, side == 0 ? nullptr : syn, stream);
  if (rc != LEAD_OK) {
    cleanup();
    return rc;
  }
  lead_decode_opts o{};
  o.side = side;
  o.use_lead = 1;
  o.max_iter = 32;
  o.precision = prec;
  o.alpha = 1.0f;
  o.p = p;
  o.estimator = LEAD_EST_EXACT;
  auto time_current = [&](float* ms) -> int {
    int r = lead_decode(code, &o, syn, shots, corr, st, nullptr, nullptr, ws, wsb, stream);     // warm-up
    if (r != LEAD_OK) return r;
    if (cudaEventRecord(e0, stream) != cudaSuccess) return LEAD_ECUDA;
    for (int k = 0; k < 2 && r == LEAD_OK; ++k) r = lead_decode(code, &o, syn, shots, corr, st, nullptr, nullptr, ws, wsb, stream);
    if (r != LEAD_OK) return r;
    if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return LEAD_ECUDA;
    *ms *= 0.5f;
    return LEAD_OK;
  };
  // one launch shape: the kernel, its geometry and its partner table (null: the default one)
  struct Cand {
    TunedKernel k;
    int minblocks = -1;
    long spill = 0;
    float ms = 0.0f;
    std::vector<char> cubin;
  };
  // every candidate is timed as the only tuned shape (the default kernel: none); the list of
  // shapes tuned before is put back afterwards
  std::vector<TunedKernel> saved;
  saved.swap(ds.tuned[prec]);
  std::vector<Cand> cands;
  {
    Cand c;                                   // the default kernel
    c.k.p = p;
    c.k.lib = ds.bp_module[prec];
    c.k.func = ds.bp_func[prec];
    c.k.per_sm = ds.bp_per_sm[prec];
    c.k.block = hs.bp_block;
    c.k.spb = hs.bp_spb;
    c.k.cluster = hs.bp_cluster;
    c.k.maxreg = hs.bp_maxreg[prec];
    c.k.smem = hs.bp_smem[prec];
    rc = time_current(&c.ms);
    cands.push_back(std::move(c));
  }
  // launch shapes: (shots per CTA, cluster size)
  std::vector<std::pair<int, int>> shapes;
  if (hs.bp_cluster == 1) {
    for (int f = 1; f <= 4; ++f) shapes.push_back({hs.bp_spb * f, 1});
  } else {
    // the default, and the sizes that leave few idle lanes in the last warp of a CTA for the
    // codes here (a cluster is at most 8 CTAs, the portable limit)
    shapes.push_back({1, hs.bp_cluster});
    for (int c : {1, 2, 3, 4, 7})       // 1: the whole shot in one CTA, where its state fits
      if (c != hs.bp_cluster) shapes.push_back({1, c});
  }
  for (const auto& shape : shapes) {
    if (rc != LEAD_OK) break;
    const int spb = shape.first;
    const Geometry g = bp_geometry(code, side, prec, spb, shape.second);
    if (g.block > 1024 || g.smem > 227u * 1024u) continue;
    if (g.cluster == 1 && (size_t)code->nl * g.ts >= 32768) continue;
    if (g.cluster > 1 && (size_t)code->nl * g.ts >= 65536) continue;      // u32 table: 16-bit addresses
    for (int m = g.minblocks; m >= std::max(1, g.minblocks - 2) && rc == LEAD_OK; --m) {
      Geometry gm = g;
      gm.minblocks = m;
      Cand c;
      c.minblocks = m;
      c.k.p = p;
      c.k.owned = true;
      c.k.spb = spb;
      c.k.cluster = g.cluster;
      c.k.block = g.block;
      c.k.smem = g.smem;
      c.k.maxreg = std::min(255, (65536 / (g.block * m)) & ~7);
      if (spb == hs.bp_spb && g.cluster == hs.bp_cluster && c.k.maxreg == hs.bp_maxreg[prec]) continue;   // default
      std::string log;
      rc = nvrtc_build(prelude(code, side, gm, prec) + kLeadJitSource, c.k.maxreg, &c.cubin, &log);
      if (rc != LEAD_OK) break;
      c.spill = spill_bytes(log);
      cudaLibrary_t lib = nullptr;
      cudaKernel_t kern = nullptr;
      const char* name = g.cluster > 1 ? "lead_bp_jit_cluster" : "lead_bp_jit";
      if (cudaLibraryLoadData(&lib, c.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
          cudaLibraryGetKernel(&kern, lib, name) != cudaSuccess ||
          cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem) !=
              cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.k.per_sm, (const void*)kern, g.block, g.smem) !=
              cudaSuccess ||
          c.k.per_sm < 1) {
        if (lib) cudaLibraryUnload(lib);
        rc = LEAD_ECUDA;
        break;
      }
      c.k.lib = lib;
      c.k.func = kern;
      if (spb != hs.bp_spb || g.cluster != hs.bp_cluster) {
        // this shape's partner table (bytes: u16 entries, or u32 for the larger cluster shapes)
        const std::vector<uint8_t> pa = partner_table_bytes(code, side, g);
        if (cudaMalloc(&c.k.pa, pa.size()) != cudaSuccess ||
            cudaMemcpy(c.k.pa, pa.data(), pa.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
          release_tuned(c.k);
          rc = LEAD_EOOM;
          break;
        }
      }
      ds.tuned[prec].assign(1, c.k);          // time it as the only tuned shape
      rc = time_current(&c.ms);
      ds.tuned[prec].clear();
      cands.push_back(std::move(c));
    }
  }
  cleanup();
  ds.tuned[prec].swap(saved);
  if (rc != LEAD_OK) {
    for (Cand& c : cands) release_tuned(c.k);     // the default entry owns nothing
    return rc;
  }
  size_t best = 0;
  for (size_t i = 1; i < cands.size(); ++i)
    if (cands[i].ms < cands[best].ms) best = i;
  std::ostringstream r;
  r << "side " << side << " precision " << prec << ", " << shots << " shots at p = " << p << ":\n";
  for (size_t i = 0; i < cands.size(); ++i) {
    const Cand& c = cands[i];
    r << "  " << (i == 0 ? "default kernel: " : "");
    if (c.k.cluster > 1) r << "cluster of " << c.k.cluster << " CTAs x " << c.k.block << " threads, ";
    else r << c.k.spb << " shot(s) per CTA x " << c.k.block << " threads, ";
    if (c.minblocks > 0) r << c.minblocks << " CTA(s) per SM requested, ";
    r << "<= " << c.k.maxreg << " registers, ";
    if (c.minblocks > 0) r << c.spill << " B spilled, ";
    r << c.k.per_sm << " resident: " << c.ms << " ms" << (i == best ? "  <- kept" : "") << "\n";
  }
  if (report) *report += r.str();
  // the fastest becomes the tuned shape for p (replacing one tuned at the same p); the other
  // candidates are released
  for (size_t i = 0; i < cands.size(); ++i)
    if (i != best) release_tuned(cands[i].k);
  auto& list = ds.tuned[prec];
  for (size_t i = 0; i < list.size(); ++i)
    if (std::fabs(std::log(list[i].p / p)) < 1e-9) {
      release_tuned(list[i]);
      list.erase(list.begin() + (long)i);
      break;
    }
  list.push_back(cands[best].k);
  return LEAD_OK;
}

}  // namespace lead

extern "C" int lead_code_autotune(lead_code* code, int32_t side, int32_t precision, double p, int64_t shots,
                                  char* report, size_t report_bytes) {
  if (!code || side < 0 || side > 1 || precision < 0 || precision >= lead::kPrecModes || !(p > 0.0 && p < 0.5) ||
      shots < 1 || shots > (int64_t)1 << 24)
    return LEAD_EINVAL;
  if (code->device < 0) return LEAD_ESTATE;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return LEAD_ECUDA;
  if (cur != code->device) return LEAD_ESTATE;
  std::string msg;
  const int rc = lead::autotune_one(code, side, precision, p, shots, &msg);
  if (report && report_bytes) {
    const size_t n = std::min(report_bytes - 1, msg.size());
    std::memcpy(report, msg.data(), n);
    report[n] = '\0';
  }
  return rc;
}

extern "C" int lead_code_compile(lead_code* code, char* log, size_t log_bytes) {
  if (!code) return LEAD_EINVAL;
  std::string msg;
  int rc = LEAD_OK;
  for (int prec = 0; prec < lead::kPrecModes && rc == LEAD_OK; ++prec)
    for (int side = 0; side < 2 && rc == LEAD_OK; ++side) {
      std::lock_guard<std::mutex> lock(code->jit_mu);
      rc = lead::compile_one(code, side, prec, &msg);
    }
  if (log && log_bytes) {
    const size_t n = std::min(log_bytes - 1, msg.size());
    std::memcpy(log, msg.data(), n);
    log[n] = '\0';
  }
  return rc;
}
