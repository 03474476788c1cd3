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

Geometry bp_geometry(const lead_code* code, int side, int prec) {
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
    return msgs + sizeof(uint32_t) * ((size_t)spb * P.words_m + (size_t)spb * code->words_n + 2 * (size_t)spb + 2);
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
  s << "};\n__device__ constexpr unsigned long long kRowMask[" << P.m_l << "] = {";
  for (int r = 0; r < P.m_l; ++r) s << (r ? "," : "") << P.rowmask[r] << "ull";
  // the same rows over the two words of the kernel's hard-decision bits: local index j < 32 at
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

void jit_unload(lead_code* code) {
  for (auto& ds : code->dside)
    for (int prec = 0; prec < kPrecModes; ++prec) {
      if (ds.bp_module[prec]) cudaLibraryUnload(static_cast<cudaLibrary_t>(ds.bp_module[prec]));
      ds.bp_module[prec] = nullptr;
      ds.bp_func[prec] = nullptr;
    }
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
  const long long groups = (args.shots + hs.bp_spb - 1) / hs.bp_spb;     // shots per CTA or per cluster
  const long long units = std::max<long long>(1, ((long long)sm_count * ds.bp_per_sm[prec]) / hs.bp_cluster);
  const long long blocks = std::min<long long>(groups, units) * hs.bp_cluster;
  BPJitArgs a = args;
  void* params[] = {&a};
  if (cudaLaunchKernel(ds.bp_func[prec], dim3((unsigned)blocks), dim3(hs.bp_block), params, hs.bp_smem[prec],
                       static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LEAD_ECUDA;
  return LEAD_OK;
}

// Autotuning of one side's kernel in one precision mode: the resident CTAs per SM, i.e. the
// register cap per thread, from what shared memory allows down to at most three fewer. Every
// candidate is compiled, loaded and timed (CUDA events, one warm-up and two timed calls of
// lead_decode) on `shots` shots sampled at p; the fastest is kept for every later call. The
// geometry (slots, shots per CTA, cluster) and so every output is the same for all candidates.
int autotune_one(lead_code* code, int side, int prec, double p, int64_t shots, std::string* report) {
  HostSide& hs = code->side[side];
  DeviceSide& ds = code->dside[side];
  int rc = jit_ensure(code, side, prec);            // the default kernel, compiled and loaded
  if (rc != LEAD_OK) return rc;
  Geometry g = bp_geometry(code, side, prec);
  const int top = g.minblocks;
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
  struct Cand {
    int minblocks, maxreg, per_sm;
    long spill;
    float ms;
    std::vector<char> cubin;
    void* lib;
    void* kern;
  };
  std::vector<Cand> cands;
  // the kernel in use first (compile_one's choice), then every other occupancy
  {
    Cand c{};
    c.minblocks = -1;
    c.maxreg = hs.bp_maxreg[prec];
    c.per_sm = ds.bp_per_sm[prec];
    c.cubin = hs.bp_cubin[prec];
    c.lib = ds.bp_module[prec];
    c.kern = ds.bp_func[prec];
    rc = time_current(&c.ms);
    if (rc != LEAD_OK) {
      cleanup();
      return rc;
    }
    cands.push_back(std::move(c));
  }
  for (int m = top; m >= std::max(1, top - 3) && rc == LEAD_OK; --m) {
    Geometry gm = g;
    gm.minblocks = m;
    Cand c{};
    c.minblocks = m;
    c.maxreg = std::min(255, (65536 / (g.block * m)) & ~7);
    if (c.maxreg == hs.bp_maxreg[prec]) continue;     // the kernel in use
    std::string log;
    rc = nvrtc_build(prelude(code, side, gm, prec) + kLeadJitSource, c.maxreg, &c.cubin, &log);
    if (rc != LEAD_OK) break;
    c.spill = spill_bytes(log);
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    const char* name = hs.bp_cluster > 1 ? "lead_bp_jit_cluster" : "lead_bp_jit";
    if (cudaLibraryLoadData(&lib, c.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
        cudaLibraryGetKernel(&kern, lib, name) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs.bp_smem[prec]) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.per_sm, (const void*)kern, hs.bp_block, hs.bp_smem[prec]) !=
            cudaSuccess ||
        c.per_sm < 1) {
      if (lib) cudaLibraryUnload(lib);
      rc = LEAD_ECUDA;
      break;
    }
    c.lib = lib;
    c.kern = kern;
    // time it in place of the kernel in use
    void* old_lib = ds.bp_module[prec];
    void* old_kern = ds.bp_func[prec];
    const int old_per_sm = ds.bp_per_sm[prec];
    ds.bp_module[prec] = lib;
    ds.bp_func[prec] = kern;
    ds.bp_per_sm[prec] = c.per_sm;
    rc = time_current(&c.ms);
    ds.bp_module[prec] = old_lib;
    ds.bp_func[prec] = old_kern;
    ds.bp_per_sm[prec] = old_per_sm;
    cands.push_back(std::move(c));
  }
  cleanup();
  if (rc != LEAD_OK) {
    for (size_t i = 1; i < cands.size(); ++i) cudaLibraryUnload(static_cast<cudaLibrary_t>(cands[i].lib));
    return rc;
  }
  size_t best = 0;
  for (size_t i = 1; i < cands.size(); ++i)
    if (cands[i].ms < cands[best].ms) best = i;
  std::ostringstream r;
  r << "side " << side << " precision " << prec << ", " << shots << " shots at p = " << p << ":\n";
  for (size_t i = 0; i < cands.size(); ++i) {
    const Cand& c = cands[i];
    if (c.minblocks < 0) r << "  kernel in use, <= " << c.maxreg << " registers (" << c.per_sm << " resident)";
    else r << "  " << c.minblocks << " CTA(s) per SM, <= " << c.maxreg << " registers, " << c.spill
           << " B spilled (" << c.per_sm << " resident)";
    r << ": " << c.ms << " ms" << (i == best ? "  <- kept" : "") << "\n";
  }
  if (report) *report += r.str();
  // keep the fastest; unload the others (including the kernel in use if it lost)
  for (size_t i = 0; i < cands.size(); ++i)
    if (i != best) cudaLibraryUnload(static_cast<cudaLibrary_t>(cands[i].lib));
  ds.bp_module[prec] = cands[best].lib;
  ds.bp_func[prec] = cands[best].kern;
  ds.bp_per_sm[prec] = cands[best].per_sm;
  hs.bp_cubin[prec] = std::move(cands[best].cubin);
  hs.bp_maxreg[prec] = cands[best].maxreg;
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
