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
  auto smem_for = [&](int ts, int spb, size_t mb) {
    const size_t msgs = ((size_t)ts * code->nl * 3 * mb + 15) & ~size_t(15);
    return msgs + sizeof(uint32_t) * ((size_t)spb * P.words_m + (size_t)spb * code->words_n + 2 * (size_t)spb);
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
  g.block = (g.ts + 31) / 32 * 32;
  // CTAs per SM that shared memory allows (227 KB usable, 1 KB reserved per CTA), capped so
  // that each thread keeps at least 64 registers
  int by_smem = (int)((227u * 1024u) / (g.smem + 1024));
  int by_regs = 65536 / (g.block * 64);
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
    << "#define LEAD_PA16 " << (cluster_pa16(g, code->nl) ? 1 : 0) << "\n";
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

}  // namespace lead

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
