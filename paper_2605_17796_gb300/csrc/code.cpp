// Host construction of the quantum Tanner code (Sec. II-A, II-B) and the host-only ABI calls.
//
// Everything here is plain C++ that runs without a GPU: validation of the group table and of
// the generating sets (symmetry, Total No-Conjugacy), the faces and local views of the
// left-right Cayley complex, the local check rows kron(G_B, G_A) / kron(H_B, H_A), the GF(2)
// ranks of H_Z and H_X and the logical operators used by the residual check.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lead_internal.h"

namespace {

using Row = std::vector<uint64_t>;

// ---- small GF(2) matrices: rows are bit masks over at most 64 columns -----------------------

// Reduced row echelon form; pivots are the lowest column indices (the canonical basis of the
// row space). Zero rows are dropped.
std::vector<uint64_t> rref_small(std::vector<uint64_t> rows, int cols) {
  std::vector<uint64_t> out;
  size_t r = 0;
  for (int c = 0; c < cols && r < rows.size(); ++c) {
    size_t p = r;
    while (p < rows.size() && !((rows[p] >> c) & 1)) ++p;
    if (p == rows.size()) continue;
    std::swap(rows[r], rows[p]);
    for (size_t i = 0; i < rows.size(); ++i)
      if (i != r && ((rows[i] >> c) & 1)) rows[i] ^= rows[r];
    ++r;
  }
  rows.resize(r);
  return rows;
}

// Canonical (RREF) basis of the dual of the row space of `rows`.
std::vector<uint64_t> dual_small(const std::vector<uint64_t>& rows, int cols) {
  std::vector<uint64_t> R = rref_small(rows, cols);
  std::vector<int> piv;
  for (auto x : R) piv.push_back(__builtin_ctzll(x));
  std::vector<uint64_t> ker;
  for (int f = 0; f < cols; ++f) {
    if (std::find(piv.begin(), piv.end(), f) != piv.end()) continue;
    uint64_t x = 1ull << f;
    for (size_t i = 0; i < R.size(); ++i)
      if ((R[i] >> f) & 1) x |= 1ull << piv[i];
    ker.push_back(x);
  }
  return rref_small(ker, cols);
}

std::vector<uint64_t> bytes_to_masks(const uint8_t* M, int rows, int cols) {
  std::vector<uint64_t> out(rows, 0);
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j)
      if (M[i * cols + j] & 1) out[i] |= 1ull << j;
  return out;
}

std::vector<uint8_t> masks_to_bytes(const std::vector<uint64_t>& m, int cols) {
  std::vector<uint8_t> out(m.size() * cols, 0);
  for (size_t i = 0; i < m.size(); ++i)
    for (int j = 0; j < cols; ++j) out[i * cols + j] = (m[i] >> j) & 1;
  return out;
}

// Row grouping of the local code kron(R_B, R_A) (per-qubit-prior posterior, Algorithm 1 Phase 1):
// a local error E (rows a, columns b) has syndrome S = R_A F with F = (R_B x_a)_a the row images,
// so the coset of S is the set of row-image matrices F with R_A F = S, each combined with any
// row patterns of those images. Stores the class members, the least F of every syndrome and the
// F of zero syndrome; left empty where the tables would be too large.
void row_grouping(lead::HostSide& hs, const std::vector<uint64_t>& RA, const std::vector<uint64_t>& RB,
                  int delta) {
  hs.xcls.clear();
  hs.cbase.clear();
  hs.ckern.clear();
  const int kA = hs.kRA, kB = hs.kRB;
  if (delta * kB > 24 || kB >= delta) return;
  const int NX = 1 << delta, NF = 1 << kB;
  std::vector<int> fx(NX, 0);
  for (int x = 0; x < NX; ++x)
    for (int rB = 0; rB < kB; ++rB)
      if (__builtin_popcountll(RB[rB] & (uint64_t)x) & 1) fx[x] |= 1 << rB;
  for (int f = 0; f < NF; ++f) {
    size_t before = hs.xcls.size();
    for (int x = 0; x < NX; ++x)
      if (fx[x] == f) hs.xcls.push_back((uint8_t)x);
    if (hs.xcls.size() - before != (size_t)(NX / NF)) {   // R_B rank-deficient: classes uneven
      hs.xcls.clear();
      return;
    }
  }
  // bit (rB*kA + rA) of S is the parity of F over the bits a*kB + rB with RA[rA] bit a set
  std::vector<uint32_t> smask(kA * kB, 0);
  for (int rA = 0; rA < kA; ++rA)
    for (int rB = 0; rB < kB; ++rB)
      for (int a = 0; a < delta; ++a)
        if ((RA[rA] >> a) & 1) smask[rB * kA + rA] |= 1u << (a * kB + rB);
  hs.cbase.assign((size_t)1 << hs.m_l, 0xFFFFFFFFu);
  const uint32_t NFF = 1u << (delta * kB);
  for (uint32_t F = 0; F < NFF; ++F) {
    uint32_t S = 0;
    for (int r = 0; r < kA * kB; ++r) S |= (uint32_t)(__builtin_popcount(F & smask[r]) & 1) << r;
    if (hs.cbase[S] == 0xFFFFFFFFu) hs.cbase[S] = F;
    if (S == 0) hs.ckern.push_back(F);
  }
}

// ---- large GF(2) matrices: packed rows of `words` 64-bit words ------------------------------

inline bool bit(const Row& r, int c) { return (r[c >> 6] >> (c & 63)) & 1; }
inline void xor_into(Row& a, const Row& b) {
  for (size_t w = 0; w < a.size(); ++w) a[w] ^= b[w];
}

// In-place RREF; returns the pivot columns (rows beyond the rank are zero and dropped).
std::vector<int> rref_big(std::vector<Row>& rows, int cols) {
  std::vector<int> piv;
  size_t r = 0;
  for (int c = 0; c < cols && r < rows.size(); ++c) {
    size_t p = r;
    while (p < rows.size() && !bit(rows[p], c)) ++p;
    if (p == rows.size()) continue;
    std::swap(rows[r], rows[p]);
    for (size_t i = 0; i < rows.size(); ++i)
      if (i != r && bit(rows[i], c)) xor_into(rows[i], rows[r]);
    piv.push_back(c);
    ++r;
  }
  rows.resize(r);
  return piv;
}

// Representatives of ker(Hk) modulo rowspace(Hs): the logical operators that detect a residual
// in ker(Hs) outside rowspace(Hk)... see lead_check: for side 0 (X residuals checked by H_Z),
// the logicals are Z-type: a basis of ker(H_X) completed over rowspace(H_Z).
std::vector<Row> logical_basis(std::vector<Row> kernel_of, std::vector<Row> span_of, int cols,
                               int want) {
  // kernel of `kernel_of`
  std::vector<int> piv = rref_big(kernel_of, cols);
  std::vector<char> is_piv(cols, 0);
  for (int c : piv) is_piv[c] = 1;
  const size_t words = (cols + 63) / 64;
  // echelon set seeded with rowspace(span_of)
  std::vector<int> epiv = rref_big(span_of, cols);
  std::vector<Row> E = span_of;
  std::vector<Row> out;
  for (int f = 0; f < cols && (int)out.size() < want; ++f) {
    if (is_piv[f]) continue;
    Row x(words, 0);
    x[f >> 6] |= 1ull << (f & 63);
    for (size_t i = 0; i < piv.size(); ++i)
      if (bit(kernel_of[i], f)) x[piv[i] >> 6] |= 1ull << (piv[i] & 63);
    Row y = x;
    for (size_t i = 0; i < E.size(); ++i)
      if (bit(y, epiv[i])) xor_into(y, E[i]);
    bool nz = false;
    for (auto w : y) nz |= (w != 0);
    if (!nz) continue;
    // new independent direction: keep x (a true kernel vector) and extend the echelon set
    int c = 0;
    while (!bit(y, c)) ++c;
    for (size_t i = 0; i < E.size(); ++i)
      if (bit(E[i], c)) xor_into(E[i], y);
    E.push_back(y);
    epiv.push_back(c);
    out.push_back(x);
  }
  return out;
}

int build(const lead_group* G, const int32_t* A, const int32_t* B, int32_t delta,
          const uint8_t* GA, int32_t kA, const uint8_t* GB, int32_t kB, lead_code* code) {
  if (!G || !G->mul || !A || !B || !GA) return LEAD_EINVAL;
  const int order = G->order;
  if (order < 1 || order > 4096 || delta < 2 || delta > lead::kMaxDelta) return LEAD_EINVAL;
  if (kA < 1 || kA >= delta) return LEAD_EINVAL;
  const int nl = delta * delta;
  code->order = order;
  code->delta = delta;
  code->nl = nl;
  code->mul.assign(G->mul, G->mul + (size_t)order * order);
  for (int x : code->mul)
    if (x < 0 || x >= order) return LEAD_ENOTGROUP;
  const auto& mul = code->mul;
  // identity: the element e with e x = x for all x
  int e = -1;
  for (int i = 0; i < order && e < 0; ++i) {
    bool ok = true;
    for (int x = 0; x < order && ok; ++x) ok = mul[i * order + x] == x && mul[x * order + i] == x;
    if (ok) e = i;
  }
  if (e < 0) return LEAD_ENOTGROUP;
  code->identity = e;
  code->inv.assign(order, -1);
  for (int i = 0; i < order; ++i)
    for (int j = 0; j < order; ++j)
      if (mul[i * order + j] == e) { code->inv[i] = j; break; }
  for (int i = 0; i < order; ++i)
    if (code->inv[i] < 0 || mul[code->inv[i] * order + i] != e) return LEAD_ENOTGROUP;
  // rows and columns must be permutations (Latin square)
  {
    std::vector<int> seen(order);
    for (int i = 0; i < order; ++i) {
      std::fill(seen.begin(), seen.end(), 0);
      for (int j = 0; j < order; ++j) if (seen[mul[i * order + j]]++) return LEAD_ENOTGROUP;
      std::fill(seen.begin(), seen.end(), 0);
      for (int j = 0; j < order; ++j) if (seen[mul[j * order + i]]++) return LEAD_ENOTGROUP;
    }
  }
  // generating sets (Sec. II-A): symmetric, no repeats, no identity
  code->A.assign(A, A + delta);
  code->B.assign(B, B + delta);
  for (const auto* S : {&code->A, &code->B}) {
    for (int i = 0; i < delta; ++i) {
      int x = (*S)[i];
      if (x < 0 || x >= order) return LEAD_EINVAL;
      if (x == e) return LEAD_ENOTSYM;
      for (int j = 0; j < i; ++j) if ((*S)[j] == x) return LEAD_ENOTSYM;
    }
    for (int i = 0; i < delta; ++i)
      if (std::find(S->begin(), S->end(), code->inv[(*S)[i]]) == S->end()) return LEAD_ENOTSYM;
  }
  // Total No-Conjugacy: a g != g b for all a, b, g
  for (int g = 0; g < order; ++g)
    for (int a : code->A)
      for (int b : code->B)
        if (mul[a * order + g] == mul[g * order + b]) return LEAD_ENOTTNC;
  std::vector<int> ainv(delta), binv(delta);
  for (int i = 0; i < delta; ++i) {
    ainv[i] = int(std::find(code->A.begin(), code->A.end(), code->inv[code->A[i]]) - code->A.begin());
    binv[i] = int(std::find(code->B.begin(), code->B.end(), code->inv[code->B[i]]) - code->B.begin());
  }

  // local codes (Sec. II-B); missing G_B means C_B = C_A^perp
  std::vector<uint64_t> gA = bytes_to_masks(GA, kA, delta);
  if ((int)rref_small(gA, delta).size() != kA) return LEAD_EINVAL;
  std::vector<uint64_t> gB;
  if (GB) {
    if (kB < 1 || kB >= delta) return LEAD_EINVAL;
    gB = bytes_to_masks(GB, kB, delta);
    if ((int)rref_small(gB, delta).size() != kB) return LEAD_EINVAL;
  } else {
    gB = dual_small(gA, delta);
  }
  std::vector<uint64_t> hA = dual_small(gA, delta);
  std::vector<uint64_t> hB = dual_small(gB, delta);
  code->kA = kA;
  code->kB = (int)gB.size();
  code->GA = masks_to_bytes(gA, delta);
  code->GB = masks_to_bytes(gB, delta);
  code->HA = masks_to_bytes(hA, delta);
  code->HB = masks_to_bytes(hB, delta);

  // faces: (g, a, b) ~ (a g b, a^-1, b^-1); the qubit is the lexicographically smaller tuple
  auto twin = [&](int g, int ia, int ib, int* tg, int* ta, int* tb) {
    *tg = mul[mul[code->A[ia] * order + g] * order + code->B[ib]];
    *ta = ainv[ia];
    *tb = binv[ib];
  };
  std::vector<int32_t> qid((size_t)order * nl, -1);
  auto tix = [&](int g, int ia, int ib) { return ((size_t)g * delta + ia) * delta + ib; };
  int n = 0;
  for (int g = 0; g < order; ++g)
    for (int ia = 0; ia < delta; ++ia)
      for (int ib = 0; ib < delta; ++ib) {
        int tg, ta, tb;
        twin(g, ia, ib, &tg, &ta, &tb);
        if (tix(g, ia, ib) < tix(tg, ta, tb)) qid[tix(g, ia, ib)] = n++;
      }
  for (int g = 0; g < order; ++g)
    for (int ia = 0; ia < delta; ++ia)
      for (int ib = 0; ib < delta; ++ib)
        if (qid[tix(g, ia, ib)] < 0) {
          int tg, ta, tb;
          twin(g, ia, ib, &tg, &ta, &tb);
          qid[tix(g, ia, ib)] = qid[tix(tg, ta, tb)];
        }
  if (n * 2 != order * nl) return LEAD_ENOTTNC;
  code->n = n;
  code->words_n = ((n + 31) / 32 + 3) / 4 * 4;
  const int words64 = (n + 63) / 64;

  std::vector<Row> Hrows[2];
  for (int s = 0; s < 2; ++s) {
    lead::HostSide& hs = code->side[s];
    const auto& RA = (s == 0) ? gA : hA;
    const auto& RB = (s == 0) ? gB : hB;
    hs.kRA = (int)RA.size();
    hs.kRB = (int)RB.size();
    hs.RA = masks_to_bytes(RA, delta);
    hs.RB = masks_to_bytes(RB, delta);
    hs.m_l = hs.kRA * hs.kRB;
    if (hs.m_l < 1 || hs.m_l > lead::kMaxLocalRows) return LEAD_EINVAL;
    hs.m = order * hs.m_l;
    // local rows r = rB * kRA + rA of kron(RB, RA) over j = ib * delta + ia
    hs.rowmask.assign(hs.m_l, 0);
    hs.max_row_weight = 0;
    for (int rB = 0; rB < hs.kRB; ++rB)
      for (int rA = 0; rA < hs.kRA; ++rA) {
        uint64_t msk = 0;
        for (int ib = 0; ib < delta; ++ib)
          for (int ia = 0; ia < delta; ++ia)
            if (((RB[rB] >> ib) & 1) && ((RA[rA] >> ia) & 1)) msk |= 1ull << (ib * delta + ia);
        hs.rowmask[rB * hs.kRA + rA] = msk;
        hs.max_row_weight = std::max(hs.max_row_weight, __builtin_popcountll(msk));
      }
    if (hs.max_row_weight > lead::kMaxSupport) return LEAD_EINVAL;
    row_grouping(hs, RA, RB, delta);
    // views
    hs.views.assign((size_t)order * nl, 0);
    for (int v = 0; v < order; ++v)
      for (int ia = 0; ia < delta; ++ia)
        for (int ib = 0; ib < delta; ++ib) {
          int j = ib * delta + ia;
          int q = (s == 0) ? qid[tix(v, ia, ib)]
                           : qid[tix(mul[code->A[ia] * order + v], ainv[ia], ib)];
          hs.views[(size_t)v * nl + j] = q;
        }
    // the two views of every qubit (vertex order), partner slots
    std::vector<int32_t> cnt(n, 0);
    hs.qslots.assign((size_t)n * 2, 0);
    for (int v = 0; v < order; ++v)
      for (int j = 0; j < nl; ++j) {
        int q = hs.views[(size_t)v * nl + j];
        if (cnt[q] >= 2) return LEAD_ENOTTNC;
        hs.qslots[(size_t)q * 2 + cnt[q]++] = (uint32_t)(v * nl + j);
      }
    hs.partner.assign((size_t)order * nl, 0);
    for (int q = 0; q < n; ++q) {
      if (cnt[q] != 2) return LEAD_ENOTTNC;
      uint32_t a = hs.qslots[(size_t)q * 2], b = hs.qslots[(size_t)q * 2 + 1];
      if (a / nl == b / nl) return LEAD_ENOTTNC;
      hs.partner[a] = b | 0x80000000u;     // a has the smaller vertex: it is the first view
      hs.partner[b] = a;
    }
    // kernel parameters
    lead::SideParams& P = hs.params;
    std::memset(&P, 0, sizeof(P));
    P.order = order;
    P.nl = nl;
    P.m_l = hs.m_l;
    P.m = hs.m;
    P.words_m = ((hs.m + 31) / 32 + 3) / 4 * 4;
    for (int r = 0; r < hs.m_l; ++r) {
      P.rowmask[r] = hs.rowmask[r];
      int k = 0;
      for (int j = 0; j < nl; ++j)
        if ((hs.rowmask[r] >> j) & 1) P.supp[r][k++] = (uint8_t)j;
      P.supp_len[r] = k;
    }
    // check matrix rows (packed) for ranks and logicals
    Hrows[s].assign(hs.m, Row(words64, 0));
    for (int v = 0; v < order; ++v)
      for (int r = 0; r < hs.m_l; ++r) {
        Row& row = Hrows[s][(size_t)v * hs.m_l + r];
        for (int j = 0; j < nl; ++j)
          if ((hs.rowmask[r] >> j) & 1) {
            int q = hs.views[(size_t)v * nl + j];
            row[q >> 6] ^= 1ull << (q & 63);
          }
      }
  }
  // CSS condition H_X H_Z^T = 0 (Sec. II-B): every X row is orthogonal to every Z row
  for (const Row& x : Hrows[1])
    for (const Row& z : Hrows[0]) {
      int par = 0;
      for (int w = 0; w < words64; ++w) par ^= __builtin_popcountll(x[w] & z[w]) & 1;
      if (par) return LEAD_ECSS;
    }
  for (int s = 0; s < 2; ++s) {
    std::vector<Row> tmp = Hrows[s];
    code->side[s].rank = (int)rref_big(tmp, n).size();
  }
  code->k = n - code->side[0].rank - code->side[1].rank;
  // logicals: side 0 checks X residuals against Z-type logicals = ker(H_X) mod rowspace(H_Z);
  // side 1 checks Z residuals against X-type logicals = ker(H_Z) mod rowspace(H_X)
  for (int s = 0; s < 2; ++s) {
    std::vector<Row> L = logical_basis(Hrows[1 - s], Hrows[s], n, code->k);
    if ((int)L.size() != code->k) return LEAD_ECSS;
    auto& out = code->side[s].logicals;
    out.assign((size_t)code->k * code->words_n, 0);
    for (int i = 0; i < code->k; ++i)
      for (int q = 0; q < n; ++q)
        if (bit(L[i], q)) out[(size_t)i * code->words_n + (q >> 5)] |= 1u << (q & 31);
  }
  return LEAD_OK;
}

}  // namespace

extern "C" {

int lead_build_code(const lead_group* G, const int32_t* A, const int32_t* B, int32_t delta,
                    const uint8_t* GA, int32_t kA, const uint8_t* GB, int32_t kB,
                    lead_code** out) {
  if (!out) return LEAD_EINVAL;
  *out = nullptr;
  lead_code* code = new (std::nothrow) lead_code();
  if (!code) return LEAD_EOOM;
  int rc;
  try {
    rc = build(G, A, B, delta, GA, kA, GB, kB, code);
  } catch (const std::bad_alloc&) {
    rc = LEAD_EOOM;
  }
  if (rc != LEAD_OK) {
    delete code;
    return rc;
  }
  *out = code;
  return LEAD_OK;
}

int lead_code_get_info(const lead_code* code, lead_code_info* out) {
  if (!code || !out) return LEAD_EINVAL;
  out->n = code->n;
  out->order = code->order;
  out->delta = code->delta;
  out->k_A = code->kA;
  out->k_B = code->kB;
  for (int s = 0; s < 2; ++s) {
    out->m_l[s] = code->side[s].m_l;
    out->m[s] = code->side[s].m;
    out->rank[s] = code->side[s].rank;
    out->words_m[s] = code->side[s].params.words_m;
    out->max_row_weight[s] = code->side[s].max_row_weight;
  }
  out->k = code->k;
  out->words_n = code->words_n;
  out->prepared_device = code->device;
  return LEAD_OK;
}

int lead_code_get_views(const lead_code* code, int32_t side, int32_t* views) {
  if (!code || !views || side < 0 || side > 1) return LEAD_EINVAL;
  const auto& v = code->side[side].views;
  std::copy(v.begin(), v.end(), views);
  return LEAD_OK;
}

int lead_code_get_check_matrix(const lead_code* code, int32_t side, uint8_t* H) {
  if (!code || !H || side < 0 || side > 1) return LEAD_EINVAL;
  const auto& hs = code->side[side];
  const int nl = code->nl;
  std::memset(H, 0, (size_t)hs.m * code->n);
  for (int v = 0; v < code->order; ++v)
    for (int r = 0; r < hs.m_l; ++r)
      for (int j = 0; j < nl; ++j)
        if ((hs.rowmask[r] >> j) & 1) H[((size_t)v * hs.m_l + r) * code->n + hs.views[(size_t)v * nl + j]] ^= 1;
  return LEAD_OK;
}

void lead_free_code(lead_code* code) {
  if (!code) return;
  lead::release_device(code);
  delete code;
}

const char* lead_status_string(int status) {
  switch (status) {
    case LEAD_OK: return "ok";
    case LEAD_EINVAL: return "invalid argument, size or layout";
    case LEAD_ENOTTNC: return "generating sets violate Total No-Conjugacy";
    case LEAD_ENOTSYM: return "generating set not symmetric, repeated, or contains the identity";
    case LEAD_ECSS: return "construction violates H_X H_Z^T = 0";
    case LEAD_EOOM: return "out of memory";
    case LEAD_ECUDA: return "CUDA runtime error";
    case LEAD_ETIMEOUT: return "bounded device wait expired";
    case LEAD_ESTATE: return "code not prepared on this device";
    case LEAD_ENOTGROUP: return "table is not a group table";
    case LEAD_ECHECK: return "checked build: a kernel index failed its bounds check";
    default: return "unknown status";
  }
}

}  // extern "C"
