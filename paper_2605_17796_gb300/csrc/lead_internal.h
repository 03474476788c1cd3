// Internal definitions shared by the host construction (code.cpp) and the CUDA translation
// units of the LEAD library. Not part of the public ABI (include/lead.h is).
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lead.h"

namespace lead {

constexpr int kMaxDelta = 6;          // local views of at most 36 qubits (64-bit masks)
constexpr int kMaxLocalRows = 12;     // m_l <= 12 local checks per vertex (2^m_l-entry tables)
constexpr int kMaxSupport = 26;       // local check rows of weight <= 26 (packed sign bits)
constexpr int kMaxIter = 64;
constexpr int kPrecModes = 3;         // LEAD_PREC_FP32, LEAD_PREC_BF16, LEAD_PREC_FP16

// Per-side structure that kernels receive by value.
struct SideParams {
  int32_t order;          // vertices of the side (= |G|)
  int32_t nl;             // delta^2
  int32_t m_l;            // local rows per vertex
  int32_t m;              // global checks
  int32_t words_m;        // syndrome words per shot
  int32_t supp_len[kMaxLocalRows];
  uint8_t supp[kMaxLocalRows][kMaxSupport];   // local indices j of row r, increasing
  uint64_t rowmask[kMaxLocalRows];            // bit j set iff row r touches local index j
};

// A launch shape of the min-sum kernel kept by lead_code_autotune for calls whose prior is
// nearest (log scale) to p: its own compiled kernel and, when its shots per CTA or cluster size
// differ from the default geometry's, its own partner table.
struct TunedKernel {
  double p = 0.0;
  void* lib = nullptr;          // cudaLibrary_t; not owned when it is the default kernel
  void* func = nullptr;         // cudaKernel_t
  bool owned = false;
  int per_sm = 0, block = 0, spb = 1, cluster = 1, maxreg = 0;
  size_t smem = 0;
  uint16_t* pa = nullptr;       // owned partner table, or null for the default one
};

struct DeviceSide {
  uint16_t* views = nullptr;     // order*nl qubit ids
  uint32_t* partner = nullptr;   // order*nl: (other slot) | (this view is the first << 31)
  uint32_t* qslots = nullptr;    // n*2: slot of the qubit's first view, second view
  int32_t* enumN = nullptr;      // 2^m_l x (nl+1)
  int32_t* enumN1 = nullptr;     // 2^m_l x nl x (nl+1)
  uint64_t* ml = nullptr;        // 2^m_l least-weight coset members
  uint32_t* logicals = nullptr;  // k x words_n
  uint16_t* bp_pa = nullptr;     // partner table of the min-sum kernel (u16 entries, or u32 with
                                 // the owner rank for cluster launches)
  uint8_t* xcls = nullptr;       // row patterns of every class f = R_B x (class-major, increasing)
  uint32_t* cbase = nullptr;     // 2^m_l: one row-image matrix F with R_A F = S per local syndrome
  uint32_t* ckern = nullptr;     // row-image matrices with R_A F = 0, increasing
  void* bp_module[kPrecModes] = {};   // cudaLibrary_t of the specialised min-sum kernel, per mode
  void* bp_func[kPrecModes] = {};     // its cudaKernel_t
  int bp_per_sm[kPrecModes] = {};     // resident CTAs per SM
  std::vector<TunedKernel> tuned[kPrecModes];   // launch shapes kept by lead_code_autotune
};

struct HostSide {
  int32_t m_l = 0;
  int32_t m = 0;
  int32_t rank = 0;
  int32_t max_row_weight = 0;
  std::vector<uint64_t> rowmask;     // m_l
  std::vector<int32_t> views;        // order*nl
  std::vector<uint32_t> partner;     // order*nl
  std::vector<uint32_t> qslots;      // n*2
  std::vector<uint32_t> logicals;    // k*words_n (operators of the other type)
  std::vector<uint8_t> RA, RB;       // row factors: local checks = kron(RB, RA)
  int32_t kRA = 0, kRB = 0;
  // Row grouping of the local code (per-qubit-prior posterior): F packs f_a = R_B x_a at bits
  // a*kRB; empty when delta*kRB > 24 or R_B is rank-deficient.
  std::vector<uint8_t> xcls;
  std::vector<uint32_t> cbase, ckern;
  SideParams params{};
  std::vector<char> bp_cubin[kPrecModes];   // specialised min-sum kernel per mode (NVRTC output)
  int bp_block = 0, bp_spb = 0, bp_cluster = 1;   // the default geometry (binary32 footprint)
  size_t bp_smem[kPrecModes] = {};
  int bp_maxreg[kPrecModes] = {};          // register cap per thread it was compiled with
};

}  // namespace lead

struct lead_code {
  int32_t order = 0, delta = 0, nl = 0, kA = 0, kB = 0, n = 0, k = 0, words_n = 0;
  std::vector<int32_t> mul, inv;
  int32_t identity = -1;
  std::vector<int32_t> A, B;
  std::vector<uint8_t> GA, GB, HA, HB;    // row-major, delta columns
  lead::HostSide side[2];
  int32_t device = -1;
  lead::DeviceSide dside[2];
  unsigned long long* d_check = nullptr;   // checked build: {failures, site, index, bound}; then the
                                           // device error flags (lead_code_device_errors) in word 4
  mutable unsigned long long last_check[4] = {};   // the last record a call returned LEAD_ECHECK for
  std::mutex jit_mu;                 // guards the lazily compiled kernels of the 16-bit modes
};

namespace lead {
// Implemented in the CUDA translation units.
int prepare_device(lead_code* code, int device);
void release_device(lead_code* code);
int bp_shots_per_block(const lead_code* code);   // shots per CTA of the min-sum kernel
size_t decode_workspace_bytes(const lead_code* code, int side);   // what lead_decode reads
// Checked build: wait for the stream and turn a recorded bounds failure into LEAD_ECHECK (the
// record moves to code->last_check). Release build: LEAD_OK at once.
int check_result(const lead_code* code, void* stream);
int priors_check(const lead_code* code, const lead_decode_opts* o);   // lead_decode_priors' argument checks
struct BPJitArgs;
struct Geometry {               // launch geometry of the min-sum kernel for one side
  int spb, cluster, ts, block, minblocks;
  size_t smem;
  bool alias;                   // one shot per CTA: syndromes and correction bits share the
                                // message arrays (see bp_geometry)
};
// spb > 0 asks for that many shots per CTA instead of the default (one-CTA shots only);
// cluster >= 1 for that cluster size (shots split over a cluster only; 1 = one CTA per shot).
Geometry bp_geometry(const lead_code* code, int side, int prec = LEAD_PREC_FP32, int spb = 0, int cluster = 0);
// The u16 partner table of a one-CTA geometry: entry [j][t] = shared-memory word of the partner
// slot of (j, t) | first view << 15, t = shot sl * order + vertex v.
std::vector<uint16_t> single_cta_partner_table(const lead_code* code, int side, const Geometry& g);
// The partner table of any geometry as the bytes the kernel reads: the one-CTA table above, or
// for a cluster (indexed [j][v], v the global vertex) partner word address inside its owner CTA
// | owner rank << 13 | first << 15 as u16 when cluster_pa16, else address | rank << 16 |
// first << 31 as u32.
std::vector<uint8_t> partner_table_bytes(const lead_code* code, int side, const Geometry& g);
// Cluster launches whose slot addresses fit 13 bits and owner ranks 2 bits use a u16 partner
// table (address | owner << 13 | first << 15): half the bytes of the u32 form, so it stays in L1.
inline bool cluster_pa16(const Geometry& g, int nl) { return g.cluster > 1 && g.cluster <= 4 && nl * g.ts < 8192; }
int jit_compile(lead_code* code, std::string* log);      // binary32 kernels of both sides
int compile_one(lead_code* code, int side, int prec, std::string* log);
int jit_load(lead_code* code);
int jit_ensure(const lead_code* code, int side, int prec);   // compile + load one mode on first use
void jit_unload(lead_code* code);
int jit_launch_bp(const lead_code* code, int side, int prec, const BPJitArgs& args, int sm_count, void* stream);
}  // namespace lead
