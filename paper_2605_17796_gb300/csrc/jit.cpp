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
#include <sstream>
#include <string>
#include <vector>

#include "bp_jit_args.h"
#include "lead_internal.h"
#include "lead_jit_source.inc"   // generated at build time: kLeadJitSource

namespace lead {

namespace {

}  // namespace

Geometry bp_geometry(const lead_code* code, int side) {
  const SideParams& P = code->side[side].params;
  Geometry g{};
  auto smem_for = [&](int ts, int spb) {
    return sizeof(uint32_t) * ((size_t)ts * code->nl * 3 + (size_t)spb * P.words_m + (size_t)spb * code->words_n +
                               2 * (size_t)spb);
  };
  g.spb = bp_shots_per_block(code);
  g.cluster = 1;
  g.ts = g.spb * code->order;
  g.smem = smem_for(g.ts, g.spb);
  // a shot whose state does not leave room for two CTAs per SM is split over a thread-block
  // cluster (distributed shared memory), 2, 4 or 8 CTAs
  while (g.smem > 120u * 1024u && g.cluster < 8) {
    g.cluster *= 2;
    g.spb = 1;
    g.ts = (code->order + g.cluster - 1) / g.cluster;
    g.smem = smem_for(g.ts, 1);
  }
  g.block = (g.ts + 31) / 32 * 32;
  // CTAs per SM that shared memory allows (227 KB usable, 1 KB reserved per CTA), capped so
  // that each thread keeps at least 64 registers
  int by_smem = (int)((227u * 1024u) / (g.smem + 1024));
  int by_regs = 65536 / (g.block * 64);
  g.minblocks = std::max(1, std::min(by_smem, by_regs));
  return g;
}

namespace {

std::string prelude(const lead_code* code, int side, const Geometry& g) {
  const SideParams& P = code->side[side].params;
  int kmax = 1;
  for (int r = 0; r < P.m_l; ++r) kmax = std::max(kmax, P.supp_len[r]);
  std::ostringstream s;
  s << "#define LEAD_NL " << code->nl << "\n"
    << "#define LEAD_ML " << P.m_l << "\n"
    << "#define LEAD_TS " << g.ts << "\n"
    << "#define LEAD_BLOCK " << g.block << "\n"
    << "#define LEAD_MINBLOCKS " << g.minblocks << "\n"
    << "#define LEAD_KMAX " << kmax << "\n"
    << "#define LEAD_SPB " << g.spb << "\n"
    << "#define LEAD_CLUSTER " << g.cluster << "\n"
    << "namespace lead_jit {\n";
  s << "__device__ constexpr int kLen[" << P.m_l << "] = {";
  for (int r = 0; r < P.m_l; ++r) s << (r ? "," : "") << P.supp_len[r];
  s << "};\n__device__ constexpr int kSupp[" << P.m_l << "][" << kmax << "] = {";
  for (int r = 0; r < P.m_l; ++r) {
    s << (r ? ",{" : "{");
    for (int k = 0; k < kmax; ++k) s << (k ? "," : "") << (k < P.supp_len[r] ? (int)P.supp[r][k] : 0);
    s << "}";
  }
  // kFirst[r][k]: row r is the first local row (in increasing order) that touches slot supp[r][k]
  s << "};\n__device__ constexpr bool kFirst[" << P.m_l << "][" << kmax << "] = {";
  for (int r = 0; r < P.m_l; ++r) {
    s << (r ? ",{" : "{");
    for (int k = 0; k < kmax; ++k) {
      bool first = false;
      if (k < P.supp_len[r]) {
        const int j = P.supp[r][k];
        first = true;
        for (int r2 = 0; r2 < r; ++r2)
          if ((P.rowmask[r2] >> j) & 1) first = false;
      }
      s << (k ? "," : "") << (first ? "true" : "false");
    }
    s << "}";
  }
  s << "};\n__device__ constexpr unsigned long long kRowMask[" << P.m_l << "] = {";
  for (int r = 0; r < P.m_l; ++r) s << (r ? "," : "") << P.rowmask[r] << "ull";
  s << "};\n}\n";
  return s.str();
}

}  // namespace

int jit_compile(lead_code* code, std::string* log_out) {
  for (int side = 0; side < 2; ++side) {
    HostSide& hs = code->side[side];
    if (!hs.bp_cubin.empty()) continue;
    const Geometry g = bp_geometry(code, side);
    if (g.block > 1024 || (size_t)code->nl * g.ts >= 32768 || g.smem > 227u * 1024u) return LEAD_EINVAL;
    const std::string src = prelude(code, side, g) + kLeadJitSource;
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "lead_bp_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
      return LEAD_ECUDA;
    // LEAD_JIT_PTXAS_VERBOSE=1 adds the assembler's register / spill report to the log
    const char* verbose = std::getenv("LEAD_JIT_PTXAS_VERBOSE");
    // registers per thread that let LEAD_MINBLOCKS CTAs of this size share an SM
    const int maxreg = std::min(255, (65536 / (g.block * g.minblocks)) & ~7);
    const std::string regopt = "--maxrregcount=" + std::to_string(maxreg);
    const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=false", "-lineinfo",
                          regopt.c_str(), "--ptxas-options=-v"};
    const int nopts = (verbose && verbose[0] == '1') ? 6 : 5;
    const nvrtcResult rc = nvrtcCompileProgram(prog, nopts, opts);
    size_t logn = 0;
    nvrtcGetProgramLogSize(prog, &logn);
    std::string log(logn, '\0');
    if (logn) nvrtcGetProgramLog(prog, &log[0]);
    if (log_out) {
      std::ostringstream gs;
      gs << "side " << side << ": " << (g.cluster > 1 ? "cluster of " : "") << g.cluster << " CTA(s) x "
         << g.block << " threads, " << g.ts << " slots per CTA row, " << g.spb << " shot(s) per CTA, "
         << g.smem << " B shared memory, " << g.minblocks << " CTA(s) per SM, <= " << maxreg
         << " registers\n";
      *log_out += gs.str() + log;
    }
    if (rc != NVRTC_SUCCESS) {
      nvrtcDestroyProgram(&prog);
      return LEAD_ECUDA;
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    hs.bp_cubin.resize(n);
    nvrtcGetCUBIN(prog, hs.bp_cubin.data());
    nvrtcDestroyProgram(&prog);
    hs.bp_block = g.block;
    hs.bp_smem = g.smem;
    hs.bp_spb = g.spb;
    hs.bp_cluster = g.cluster;
  }
  return LEAD_OK;
}

int jit_load(lead_code* code) {
  for (int side = 0; side < 2; ++side) {
    HostSide& hs = code->side[side];
    DeviceSide& ds = code->dside[side];
    if (ds.bp_func) continue;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    if (cudaLibraryLoadData(&lib, hs.bp_cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess)
      return LEAD_ECUDA;
    int per_sm = 0;
    const char* name = hs.bp_cluster > 1 ? "lead_bp_jit_cluster" : "lead_bp_jit";
    if (cudaLibraryGetKernel(&kern, lib, name) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs.bp_smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)kern, hs.bp_block, hs.bp_smem) !=
            cudaSuccess ||
        per_sm < 1) {
      cudaLibraryUnload(lib);
      return LEAD_ECUDA;
    }
    ds.bp_module = lib;
    ds.bp_func = kern;
    ds.bp_per_sm = per_sm;
  }
  return LEAD_OK;
}

void jit_unload(lead_code* code) {
  for (auto& ds : code->dside) {
    if (ds.bp_module) cudaLibraryUnload(static_cast<cudaLibrary_t>(ds.bp_module));
    ds.bp_module = nullptr;
    ds.bp_func = nullptr;
  }
}

int jit_launch_bp(const lead_code* code, int side, const BPJitArgs& args, int sm_count, void* stream) {
  const HostSide& hs = code->side[side];
  const DeviceSide& ds = code->dside[side];
  if (!ds.bp_func) return LEAD_ESTATE;
  const long long groups = (args.shots + hs.bp_spb - 1) / hs.bp_spb;     // shots per CTA or per cluster
  const long long units = std::max<long long>(1, ((long long)sm_count * ds.bp_per_sm) / hs.bp_cluster);
  const long long blocks = std::min<long long>(groups, units) * hs.bp_cluster;
  BPJitArgs a = args;
  void* params[] = {&a};
  if (cudaLaunchKernel(ds.bp_func, dim3((unsigned)blocks), dim3(hs.bp_block), params, hs.bp_smem,
                       static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LEAD_ECUDA;
  return LEAD_OK;
}

}  // namespace lead

extern "C" int lead_code_compile(lead_code* code, char* log, size_t log_bytes) {
  if (!code) return LEAD_EINVAL;
  std::string msg;
  const int rc = lead::jit_compile(code, &msg);
  if (log && log_bytes) {
    const size_t n = std::min(log_bytes - 1, msg.size());
    std::memcpy(log, msg.data(), n);
    log[n] = '\0';
  }
  return rc;
}
