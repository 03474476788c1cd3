// Kernel arguments of the run-time specialised min-sum kernel. Included by the host code and
// prepended (as text) to the kernel source compiled with NVRTC, so both sides share one layout.
#pragma once

namespace lead {

struct BPJitArgs {
  int n;              // qubits
  int words_n;        // uint32 words per correction row
  int words_m;        // uint32 words per syndrome row
  int spb;            // shots per CTA
  int order;          // vertices per side (|G|)
  int max_iter;       // global min-sum iterations
  int use_lead;       // 1: LEAD prior from the local table; 0: channel prior
  float alpha;        // Phase-2 scaling
  float p;            // channel marginal (baseline prior), rounded to binary32
  long long shots;
  const unsigned int* syn;
  unsigned int* corr;
  unsigned char* status;
  int* iters;
  float* llr;
  const float* table;           // 2^m_l x nl local posterior table (nullptr for the baseline)
  const unsigned char* cls;     // class (distinct-value rank) of every table entry
  const float* pair;            // K x K prior LLRs lambda(alpha (q_c0 + q_c1)/2) of class pairs
  const int* header;            // header[0] = K; 0 means no class tables: merge from `table`
  const float* lam;             // shots x n per-qubit prior LLRs; when set, the prior of every slot
  const unsigned short* pa;     // [j][t] partner shared-memory address | first view << 15
  const unsigned short* views;  // [v][j] qubit index
  unsigned long long* check;    // checked build: bounds-failure record {failures, site, index, bound}
};

}  // namespace lead
