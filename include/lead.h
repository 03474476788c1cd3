/*
 * lead.h -- C ABI of the GB300 (sm_103a) LEAD decoding library.
 *
 * LEAD ("A Local Ensemble-Assisted Parallel Decoding Framework for Quantum Tanner Codes")
 * decodes a quantum Tanner code in three phases (Algorithm 1, Sec. III-B):
 *   Phase 1  every vertex v of one side of the left-right Cayley complex estimates the error
 *            probabilities of the Delta^2 qubits of its local view from its local syndrome
 *            s_v, and boosts the bits of its local hard decision to at least 1/2;
 *   Phase 2  the two estimates of every qubit are averaged and scaled by alpha (soft-information
 *            regularisation) into a global prior;
 *   Phase 3  a global decoder (here flooding min-sum, at most max_iter iterations, with a
 *            bit-packed check H e = s after every iteration) produces the correction.
 *
 * Conventions shared by every entry point
 *  - Return value: LEAD_OK (0) or a negative LEAD_E* code; no exception crosses the ABI.
 *    lead_status_string() names a code.
 *  - Sides: side 0 decodes X errors from the H_Z syndrome (Z-generators on V0, Sec. II-B);
 *    side 1 decodes Z errors from the H_X syndrome (X-generators on V1).
 *  - Bit vectors are arrays of uint32 words, one row per shot, bit j of word w = element
 *    32 w + j. Error and correction rows have lead_code_info.words_n words, syndrome rows
 *    lead_code_info.words_m[side] words (both rounded up to a multiple of 4 words = 16 bytes);
 *    padding bits are written as 0 and must be 0 on input.
 *  - Pointers marked (dev) are device pointers of the device the code was prepared on,
 *    (host) are host pointers. The caller owns and allocates every buffer it passes; the
 *    library owns only the code object and its device tables.
 *  - stream: a cudaStream_t passed as void*; NULL means the legacy default stream. All device
 *    work of a call is enqueued on that stream and nothing synchronises with the host, except
 *    where a call says so.
 *  - Sizes and layouts the library cannot serve return LEAD_EINVAL before any device work.
 */
#ifndef LEAD_H
#define LEAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LEAD_OK         0
#define LEAD_EINVAL    -1   /* bad argument, size or layout                                    */
#define LEAD_ENOTTNC   -2   /* A, B violate Total No-Conjugacy: ag == gb for some a, b, g      */
#define LEAD_ENOTSYM   -3   /* A or B not closed under inversion, repeated, or contains 1      */
#define LEAD_ECSS      -4   /* construction produced H_X H_Z^T != 0 (internal invariant)       */
#define LEAD_EOOM      -5   /* host or device allocation failed                                */
#define LEAD_ECUDA     -6   /* a CUDA runtime call failed                                      */
#define LEAD_ETIMEOUT  -7   /* reserved for a bounded device wait that expires; no call returns
                               it, since no kernel spins on a flag (cluster kernels use the
                               hardware cluster barrier)                                      */
#define LEAD_ESTATE    -8   /* code not prepared on a device, or prepared on another device    */
#define LEAD_ENOTGROUP -9   /* the table is not a group table (identity or inverses missing)   */
#define LEAD_ECHECK   -10   /* checked build only: a kernel index failed its bounds check      */

/* noise models of lead_sample (Sec. IV-A uses depolarizing noise) */
#define LEAD_NOISE_X      0  /* i.i.d. X flips with probability p (code capacity)              */
#define LEAD_NOISE_Z      1  /* i.i.d. Z flips with probability p                               */
#define LEAD_NOISE_DEPOL  2  /* X, Y, Z each with probability p/3                               */

/* per-shot decode status bits */
#define LEAD_ST_CONVERGED 1  /* the returned correction satisfies H e = s                     */
#define LEAD_ST_MAX_ITER  2  /* no iteration up to max_iter satisfied H e = s: decoder failure */
#define LEAD_ST_OSD       4  /* the correction was replaced by ordered-statistics decoding       */

/* precision modes of lead_decode_opts.precision */
#define LEAD_PREC_FP32    0  /* binary32 priors and messages                                   */
#define LEAD_PREC_BF16    1  /* LLRs stored as bfloat16 (round to nearest even), FP32 arithmetic  */
#define LEAD_PREC_FP16    2  /* LLRs stored as IEEE binary16 (round to nearest even, saturating
                                at +-65504), FP32 arithmetic                                    */

/* local decoders of Phase 1 (lead_decode_opts.estimator) */
#define LEAD_EST_EXACT    0  /* exact posterior of the local coset, ML hard decision (default)   */
#define LEAD_EST_MINSUM   1  /* local min-sum BP, at most Delta^2 iterations (the paper's BP part) */

typedef struct lead_code lead_code;   /* opaque; immutable after lead_build_code */

/* A finite group given by its Cayley table: mul[i * order + j] = index of g_i g_j (host). */
typedef struct {
  int32_t order;
  const int32_t* mul;
} lead_group;

typedef struct {
  int32_t n;              /* qubits = |G| Delta^2 / 2 (Sec. III-C)                              */
  int32_t order;          /* |G| = |V0| = |V1|                                                   */
  int32_t delta;          /* |A| = |B|                                                           */
  int32_t k_A, k_B;       /* dimensions of C_A and C_B                                           */
  int32_t m_l[2];         /* local checks per vertex: k_A k_B (side 0), (D-k_A)(D-k_B) (side 1)  */
  int32_t m[2];           /* global checks per side = order * m_l[side]                          */
  int32_t rank[2];        /* GF(2) ranks of H_Z (side 0) and H_X (side 1)                        */
  int32_t k;              /* logical qubits n - rank[0] - rank[1]                                */
  int32_t words_n;        /* uint32 words per error / correction row                             */
  int32_t words_m[2];     /* uint32 words per syndrome row of each side                          */
  int32_t max_row_weight[2];
  int32_t prepared_device;/* device the tables live on, or -1                                    */
} lead_code_info;

/* Options of one decode call on one side. */
typedef struct {
  int32_t side;           /* 0 or 1                                                              */
  int32_t use_lead;       /* 1: Phases 1-3; 0: the standalone min-sum baseline on the channel prior */
  int32_t max_iter;       /* global min-sum iterations, 0..64                                    */
  int32_t precision;      /* LEAD_PREC_*: storage format of the LLRs (see each entry point)       */
  float   alpha;          /* Phase-2 scaling, 0 < alpha <= 1 (Sec. III-B; 1 is the default)      */
  double  p;              /* channel marginal of this side's error type, 0 < p < 1/2              */
  int32_t estimator;      /* LEAD_EST_*: the local decoder of Phase 1 (0 = exact)                 */
} lead_decode_opts;

/*
 * lead_build_code -- the quantum Tanner code of Sec. II from (G, A, B, C_A, C_B). Host only:
 * no device is touched, so it also runs on machines without a GPU.
 *  G     (host) Cayley table of the group, validated as a group table.
 *  A, B  (host) delta element indices each; their order fixes the local coordinates. Checked:
 *        A = A^{-1}, B = B^{-1}, no repeats, no identity (Sec. II-A) and Total No-Conjugacy
 *        ag != gb for all a, b, g (Eq. group_set and the paragraph after it).
 *  GA    (host) kA x delta row-major 0/1 bytes, a full-rank generator matrix of C_A.
 *  GB    (host) kB x delta generator of C_B, or NULL for C_B = C_A^perp (the paper's choice in
 *        every instance of Sec. IV and Appendix A); then kB is ignored.
 * Readings fixed by the library (the paper leaves them open):
 *  - the face of (g, a, b) is {(g,0),(ag,1),(gb,1),(agb,0)}; (g,a,b) and (agb,a^-1,b^-1) name the
 *    same face and its qubit index is the rank of the lexicographically smaller tuple
 *    (g, index(a), index(b)) among all faces;
 *  - a V0 vertex g sees face (g,a,b) at local index j = index(b)*delta + index(a); a V1 vertex h
 *    sees at j the face (a h, a^-1, b), i.e. {(h,1),(ah,0),(hb,0),(ahb,1)};
 *  - local checks: side 0 the rows of kron(G_B, G_A), side 1 the rows of kron(H_B, H_A), where
 *    H_A, H_B and a missing G_B are the reduced-row-echelon bases of the dual codes; global
 *    check index = vertex * m_l + local row (so s_v is a contiguous m_l-bit field).
 *  out   receives a new code object; release it with lead_free_code.
 * Errors: LEAD_EINVAL (sizes; delta must be 2..6, at most 12 local rows per vertex on each side,
 *        every check row weight at most 26),
 * LEAD_ENOTGROUP, LEAD_ENOTSYM, LEAD_ENOTTNC, LEAD_ECSS, LEAD_EOOM.
 */
int lead_build_code(const lead_group* G, const int32_t* A, const int32_t* B, int32_t delta,
                     const uint8_t* GA, int32_t kA, const uint8_t* GB, int32_t kB,
                     lead_code** out);

/* Fill *out with the code's sizes (host only). */
int lead_code_get_info(const lead_code* code, lead_code_info* out);

/* Copy the local views of one side: views[v * delta^2 + j] = qubit (host array of
 * order * delta^2 int32). Host only; for inspection and tests. */
int lead_code_get_views(const lead_code* code, int32_t side, int32_t* views);

/* Copy one side's check matrix as m x n row-major 0/1 bytes (host). Host only. */
int lead_code_get_check_matrix(const lead_code* code, int32_t side, uint8_t* H);

/*
 * lead_code_compile -- specialise the global min-sum kernel to this code (host only, no device
 * needed): the kernel source is compiled at run time (NVRTC, sm_103a) with the code's local
 * check supports as constants, so every loop over a check's support has a fixed trip count.
 * Compiles the kernels of both sides in every precision mode. lead_code_prepare compiles the
 * binary32 kernels when they are missing, and a decode call in a 16-bit mode compiles and loads
 * that mode's kernel on its first use; calling lead_code_compile first moves that compile time
 * (about a second per kernel) out of the device set-up and out of the first decode call (which
 * then only loads the module; make that first call outside stream capture). log (host,
 * nullable) receives the compiler log, truncated to log_bytes. Errors: LEAD_EINVAL (sizes the
 * kernel cannot serve), LEAD_ECUDA (compilation failed; see the log).
 */
int lead_code_compile(lead_code* code, char* log, size_t log_bytes);

/*
 * lead_code_autotune -- choose, by measurement, the launch shape of one side's global min-sum
 * kernel (Algorithm 1, Phase 3) in one precision mode. The paper has no counterpart: these are
 * properties of this kernel. Candidates: for codes whose shot fits one CTA, one to four times
 * the default shots per CTA; for codes whose shot is split over a thread-block cluster, clusters
 * of 2, 3, 4 and 7 CTAs and one CTA per shot (where the block stays <= 1024 threads and shared
 * memory fits: in the 16-bit modes, for the codes here); for
 * each, the resident CTAs per SM from what shared memory allows down to two fewer (the register
 * cap per thread trades against them). Each candidate is compiled, loaded and timed with CUDA
 * events (one warm-up and two timed lead_decode calls, Phases 1-3, exact
 * estimator, alpha = 1, 32 iterations) on `shots` syndromes drawn by lead_sample at p (seed
 * 0x5EED). The fastest is kept for later calls on this side and mode whose prior p is nearest
 * (on a log scale) to this p among the tuned ones: the shape that wins depends on how many
 * iterations the shots take and how unevenly (several shots per CTA wait for the slowest).
 * Tuning again at the same p replaces that entry; untuned codes use the default kernel. Every
 * candidate runs the same arithmetic on every shot, so every decode output is bit-identical
 * whichever is used.
 *  side, precision  the kernel to tune; p in (0, 1/2); 1 <= shots <= 2^24.
 *  report (host, nullable) receives one line per candidate (shots per CTA, threads, register
 *  cap, spilled bytes, resident CTAs, ms), truncated to report_bytes.
 * Allocates and frees its own device buffers and a stream; synchronises with the device. The
 * code must be prepared on the current device, and no other call may use the code meanwhile.
 * Errors: LEAD_EINVAL, LEAD_ESTATE (not prepared on the current device), LEAD_EOOM,
 * LEAD_ECUDA (compilation, loading or a launch failed; the tuned shapes are then unchanged).
 */
int lead_code_autotune(lead_code* code, int32_t side, int32_t precision, double p, int64_t shots,
                       char* report, size_t report_bytes);

/*
 * lead_code_prepare -- upload the code's tables to `device` and compute, on that device, the
 * exact local coset weight enumerators of both sides (the p-independent part of Phase 1:
 * N_s[w] = number of local patterns of weight w with local syndrome s, N1_s[j][w] those with
 * bit j set, and the least-weight member of every coset). Synchronises with the device before
 * returning. Call once, before any stream capture; later calls on the same device return
 * LEAD_OK at once. Errors: LEAD_ECUDA, LEAD_EOOM, LEAD_ESTATE (already prepared elsewhere).
 */
int lead_code_prepare(lead_code* code, int32_t device);

/*
 * lead_code_get_enumerators -- copy one side's device-computed enumerator tables to the host:
 * N (2^m_l x (delta^2+1) int32), N1 (2^m_l x delta^2 x (delta^2+1) int32) and ml
 * (2^m_l uint64, bit j = local index j of the least-weight coset member; ties broken by the
 * least row-major key sum_{a,b} E[a][b] 2^(a*delta+b)). Any output may be NULL. Synchronous.
 */
int lead_code_get_enumerators(const lead_code* code, int32_t side, int32_t* N, int32_t* N1,
                              uint64_t* ml);

void lead_free_code(lead_code* code);

/*
 * lead_sample -- noise of Sec. IV-A and its syndromes, on the device.
 *  noise        LEAD_NOISE_X, LEAD_NOISE_Z or LEAD_NOISE_DEPOL; 0 <= p < 1.
 *  shots        rows to produce; shot_offset + row is the absolute shot index.
 *  Random numbers: the uniform for qubit i of absolute shot s is word (i mod 4) of
 *  Philox4x32-10 (Salmon et al., SC'11) with counter (i div 4, s mod 2^32, s div 2^32, 0) and
 *  key (seed mod 2^32, seed div 2^32). A qubit flips (Bernoulli) iff u < floor(p 2^32); for
 *  depolarizing, u < floor(p/3 2^32) is X, < floor(2p/3 2^32) is Y, < floor(p 2^32) is Z.
 *  err_x, err_z (dev, shots x words_n) X and Z parts of the error; syn_z (dev, shots x
 *  words_m[0]) = H_Z err_x; syn_x (dev, shots x words_m[1]) = H_X err_z. Any output may be
 *  NULL (its part is then not written).
 */
int lead_sample(const lead_code* code, int32_t noise, double p, int64_t shots, uint64_t seed,
                uint64_t shot_offset, uint32_t* err_x, uint32_t* err_z, uint32_t* syn_z,
                uint32_t* syn_x, void* stream);

/*
 * lead_prior_llr -- the prior LLR of Phase 2, lambda(p) = ln((1 - p)/p), for n binary32
 * probabilities (p clamped to [2^-23, 1 - 2^-23]): llr[i] = lambda(p[i]). It is the conversion
 * every decode call applies to merged and channel probabilities. Evaluated in binary32 pairs
 * (double-float arithmetic: TwoSum, Fast2Sum, exact products by fused multiply-add) from the
 * series ln m = 2 artanh((m - 1)/(m + 1)) after reducing (1 - p)/p to 2^e m, m in
 * [sqrt(1/2), sqrt(2)); accurate to about 2^-45 before the final rounding, so llr[i] is the
 * binary32 rounding of the exact value except for inputs within that distance of a rounding
 * boundary (3 of the 184 549 377 binary32 values in [2^-23, 1/2], each 1 ulp off). Odd about
 * 1/2: lambda(1 - p) = -lambda(p) exactly, lambda(1/2) = 0.
 *  p, llr (dev, n floats). n == 0 is a no-op. Errors: LEAD_EINVAL (n < 0, NULL pointers),
 *  LEAD_ECUDA.
 */
int lead_prior_llr(const float* p, float* llr, int64_t n, void* stream);

/* Bytes of device workspace lead_local_estimate / lead_decode need for these options
 * (16-byte aligned start required); 0 for the baseline (use_lead = 0). A multiple of 256.
 * Both calls write the local posterior table (2^m_l * Delta^2 floats, rounded up to 256 bytes)
 * and then its class tables (the class byte of every entry and the prior LLR of every pair of
 * distinct table values), and read them back. */
size_t lead_workspace_bytes(const lead_code* code, const lead_decode_opts* opts, int64_t shots);

/*
 * lead_local_table -- Phase 1 for a uniform channel prior p, for every local syndrome:
 * table[s * delta^2 + j] (dev, 2^m_l x delta^2 float) = binary32 rounding of the exact posterior
 * q_{s,j} = P(e_j = 1 | H_v e = s) = N1_s,j(r) / N_s(r) with r = p/(1-p) (both polynomials
 * evaluated in binary64 by Horner's rule), then max(q, 1/2) on the bits of the least-weight
 * coset member (the confidence boost of Algorithm 1). 0 < p < 1/2.
 */
int lead_local_table(const lead_code* code, int32_t side, double p, float* table, void* stream);

/*
 * lead_local_table_est -- the Phase-1 table of either local decoder (Alg. 1, LocalDecoder).
 * With a uniform channel prior a local decoder's output depends only on the local syndrome, so
 * every Phase-1 result of a side is one row of this 2^m_l x Delta^2 table.
 *  LEAD_EST_EXACT: as lead_local_table.
 *  LEAD_EST_MINSUM: flooding min-sum BP on the vertex's local checks (the global decoder's
 *    rules and binary32 order of operations, channel LLR lambda_f32(p) on every position), at
 *    most Delta^2 iterations (the paper runs its BP decoders up to the code length). Soft output
 *    q_j = 1/(1 + e^post_j): the binary32 posterior clamped to [-88, 88], e^x in binary64 by
 *    Cody-Waite reduction and a Taylor series with round-to-nearest operations, add and divide
 *    in binary64, one rounding to binary32. The boost max(q_j, 1/2) on the bits of the hard
 *    decision applies only when that decision satisfies the local syndrome (Alg. 1 Phase 1).
 *  iters (dev, 2^m_l int32, nullable): local iterations used per syndrome, | 1 << 16 when the
 *    local decision satisfied its syndrome (the exact estimator reports 1 | 1 << 16).
 * Errors: LEAD_EINVAL, LEAD_ESTATE, LEAD_ECUDA.
 */
int lead_local_table_est(const lead_code* code, int32_t side, double p, int32_t estimator, float* table,
                         int32_t* iters, void* stream);

/*
 * lead_local_estimate -- Phases 1 and 2 (Algorithm 1): for every qubit i with views (v0, j0)
 * and (v1, j1) on the side, p_i = alpha * ((q(s_v0, j0) + q(s_v1, j1)) * 1/2) in binary32,
 * clamped to [2^-23, 1 - 2^-23], and llr[shot * n + i] = lambda(p_i) = ln((1 - p_i)/p_i) as
 * lead_prior_llr evaluates it, then stored in the format of opts->precision:
 *   LEAD_PREC_FP32 float; LEAD_PREC_BF16 / LEAD_PREC_FP16 the 16-bit pattern (uint16) of the
 *   bfloat16 / binary16 rounding (to nearest even) of that binary32 value.
 *  syn (dev, shots x words_m[side]); llr (dev, shots x n elements of that format);
 *  workspace (dev) >= lead_workspace_bytes(opts), contents need not be initialised.
 */
int lead_local_estimate(const lead_code* code, const lead_decode_opts* opts, const uint32_t* syn,
                        int64_t shots, void* llr, void* workspace, size_t ws_bytes,
                        void* stream);

/*
 * lead_decode -- Algorithm 1 on one side for `shots` syndromes (or the standalone min-sum
 * baseline when opts->use_lead == 0, which uses the channel LLR ln((1-p)/p) for every qubit).
 *  syn    (dev, shots x words_m[side]) syndromes.
 *  corr   (dev, shots x words_n) corrections (the last hard decision when not converged).
 *  status (dev, shots uint8) LEAD_ST_* bits.
 *  iters  (dev, shots int32, nullable) global iterations used (0 = the prior's own hard decision
 *         already satisfied the syndrome).
 *  llr    (dev, shots x n float, nullable) final posterior LLRs.
 *  Global min-sum (the paper's global decoder uses BP with min-sum; OSD is not included):
 *  flooding schedule, scaling 1, binary32 arithmetic; c2v = (-1)^(s_c + #negative other v2c) *
 *  min |other v2c|, v2c = post - c2v (its sign is the IEEE sign bit), post_i = (lambda_i + U_v0)
 *  + U_v1 with U_v the sum of the messages from v's local rows in increasing row order (v0 < v1
 *  the two views of qubit i), hard decision e_i = [post_i < 0], stop at the first iteration
 *  whose decision satisfies H e = s (iteration 0 tests the prior's decision).
 *  opts->precision = LEAD_PREC_BF16 / LEAD_PREC_FP16 stores lambda_i, the c2v magnitudes (sign
 *  applied after rounding), each U_v (summed in binary32, rounded once) and post_i rounded to
 *  nearest even in that format; the hard decision reads the stored posterior. The first call
 *  in a 16-bit mode compiles (unless lead_code_compile ran) and loads that mode's kernel.
 *  Launch shape: the one lead_code_autotune kept for this side and mode at the tuned prior
 *  nearest to opts->p (log scale), else the default; the outputs do not depend on it.
 * shots == 0 is a no-op (pointers may then be NULL).
 * Errors: LEAD_EINVAL (including max_iter > 64, alpha outside (0,1] or an unknown precision;
 *        codes whose vertex count times the shared memory of one shot exceed one CTA),
 *        LEAD_ESTATE, LEAD_ECUDA.
 */
int lead_decode(const lead_code* code, const lead_decode_opts* opts, const uint32_t* syn,
                int64_t shots, uint32_t* corr, uint8_t* status, int32_t* iters, float* llr,
                void* workspace, size_t ws_bytes, void* stream);

/*
 * lead_decode_noalloc -- lead_decode without a caller-provided workspace. The paper has no
 * counterpart; this entry point exists for callers that cannot allocate device memory: a
 * real-time error-correction loop whose decode deadline leaves no room for cudaMalloc (which
 * can block and synchronise the whole device), or an application whose own pool allocator owns
 * all device memory. The per-call tables that lead_decode keeps in the workspace (the local
 * posterior table and its class tables) live instead in one fixed device array of
 * LEAD_NOALLOC_TABLE_BYTES bytes inside the library; every GPU that loads the library holds that
 * array until the process exits.
 *  Arguments and results are those of lead_decode. The call allocates nothing (no cudaMalloc,
 *  no cudaFree, no allocating library routine).
 *  The first call with shots > 0 on a device looks up the array's device address
 *  (cudaGetSymbolAddress) with that device current; make that first call before any stream
 *  capture. shots == 0 returns LEAD_OK at once, as lead_decode does.
 *  All calls on a device share the array and it keeps the last call's tables: calls whose device
 *  work overlaps (other streams, or concurrent host threads) race on it and must be serialised
 *  by the caller. Each call rewrites the tables before reading them.
 * Errors: those of lead_decode; LEAD_EINVAL also when the tables would exceed
 * LEAD_NOALLOC_TABLE_BYTES (local codes with more than 2^10 local syndromes or 36 positions).
 */
#define LEAD_NOALLOC_TABLE_BYTES 444928   /* table of 2^10 x 36 floats + class bytes + 255^2 pairs */
int lead_decode_noalloc(const lead_code* code, const lead_decode_opts* opts, const uint32_t* syn,
                        int64_t shots, uint32_t* corr, uint8_t* status, int32_t* iters,
                        float* llr, void* stream);

/*
 * Per-qubit priors. Algorithm 1 Phase 1 assumes the channel marginal p for every qubit; these
 * entry points take instead one prior probability per qubit and shot (e.g. from soft
 * measurement information), and compute the exact local posterior of every view under the
 * product of its qubits' priors:
 *   q_j = sum_{E in coset(s_v)} [E_j = 1] prod_i p_i^{E_i} (1-p_i)^{1-E_i} / (same sum without [E_j = 1]).
 * The coset is grouped by row images: a view's local error E (rows a, columns b, local index
 * j = b*Delta + a) has local syndrome R_A F with F = (R_B x_a)_a, x_a the row patterns, so
 * the sum runs over the 2^(Delta k_B - m_l) row-image matrices F of the coset and, per row, over
 * the patterns of each image. Binary32 arithmetic with log-sum-exp per row class (relative
 * error of q about 1e-5). The hard decision boosted to 1/2 (Algorithm 1 Phase 1) is the least
 * integer cost sum_j E_j W_j, W_j = rint(2^20 lambda(p_j)) with lambda the binary32 prior LLR
 * of lead_decode's decision track, ties broken by the least key sum_{a,b} E[a][b] 2^(a Delta + b).
 * Phase 2 merges the two views' boosted posteriors as lead_decode does.
 * Supported local codes: (Delta, k_B, m_l) = (6, 3, 9) and (4, 2, 4); others give LEAD_EINVAL.
 * opts->p is not used; opts->alpha, side, max_iter and use_lead are.
 *  prior (dev, shots x n float): p_i per shot and qubit, clamped to [2^-23, 1 - 2^-23].
 * The work runs in passes of at most ~256 MiB of local posteriors and prior LLRs.
 */
size_t lead_priors_workspace_bytes(const lead_code* code, const lead_decode_opts* opts, int64_t shots);

/*
 * lead_local_estimate_priors -- Phases 1-2 with per-qubit priors.
 *  llr    (dev, shots x n float) merged prior LLRs of the global decoder, binary32 in every
 *         precision mode (lead_decode_priors rounds them to the mode's format when it stores
 *         them).
 *  q_out  (dev, shots x |G| x Delta^2 float, nullable) boosted local posteriors per view
 *         ([shot][vertex][j]); when NULL, the workspace holds them one pass at a time.
 *  ml_out (dev, shots x |G| uint64, nullable) the least-cost local decision of every view
 *         (bit j = local index j).
 *  workspace (dev, 16-byte aligned) >= lead_priors_workspace_bytes(opts, shots) unless q_out.
 * Errors: LEAD_EINVAL, LEAD_ESTATE, LEAD_ECUDA.
 */
int lead_local_estimate_priors(const lead_code* code, const lead_decode_opts* opts, const uint32_t* syn,
                               int64_t shots, const float* prior, float* llr, float* q_out, uint64_t* ml_out,
                               void* workspace, size_t ws_bytes, void* stream);

/*
 * lead_decode_priors -- Algorithm 1 with per-qubit priors: Phases 1-2 as
 * lead_local_estimate_priors (opts->use_lead == 1), or the prior LLR lambda(p_i) of every qubit
 * (the standalone min-sum baseline, use_lead == 0), then lead_decode's global min-sum.
 *  Outputs as lead_decode. workspace (dev, 16-byte aligned) >= lead_priors_workspace_bytes.
 * Errors: LEAD_EINVAL, LEAD_ESTATE, LEAD_ECUDA.
 */
int lead_decode_priors(const lead_code* code, const lead_decode_opts* opts, const uint32_t* syn, int64_t shots,
                       const float* prior, uint32_t* corr, uint8_t* status, int32_t* iters, float* llr,
                       void* workspace, size_t ws_bytes, void* stream);

/*
 * lead_decode_iterated -- iterated LEAD, an extension: the paper runs Algorithm 1 once. Round 0
 * is lead_decode. Each further round takes the shots whose status lacks LEAD_ST_CONVERGED,
 * turns every qubit's last global posterior LLR post_i into a per-qubit prior
 * p_i = 1 / (1 + e^{post_i}) in binary32 (post clamped to [-17, 17], beyond which p falls
 * outside the prior clamp [2^-23, 1 - 2^-23]; e^post by Cody-Waite reduction with ln 2 split
 * as 0.693359375 + its binary32 remainder and the Taylor series of e^r through degree 7 in
 * Horner form, every operation rounded to nearest), and
 * decodes those shots again as lead_decode_priors does with that prior: the exact local
 * posterior under the product prior with use_lead == 1 (opts->estimator applies to round 0
 * only), the prior LLR alone with use_lead == 0. Shots that converged keep their result.
 *  rounds 1..64 (1 = lead_decode); stops early when every shot has converged.
 *  corr, status: those of the last round a shot ran; iters (nullable): global iterations summed
 *  over the rounds a shot ran; llr (dev, shots x n float): the posterior LLRs, required when
 *  rounds > 1 (they carry the prior from round to round).
 *  workspace (dev, 256-byte aligned) >= lead_iterated_workspace_bytes(opts, shots): the
 *  decoders' own workspace plus the compacted batch, about (4 n + 4 words_m + 4 words_n + 9)
 *  bytes per shot more.
 *  Between rounds the call copies the number of unconverged shots to the host and waits for the
 *  stream: with rounds > 1 it synchronises, so it cannot be captured in a CUDA graph.
 * Errors: those of lead_decode and lead_decode_priors (checked before round 0 when rounds > 1),
 *         LEAD_EINVAL for rounds outside 1..64, shots > 2^31 - 1 or llr NULL with rounds > 1.
 */
size_t lead_iterated_workspace_bytes(const lead_code* code, const lead_decode_opts* opts, int64_t shots);
int lead_decode_iterated(const lead_code* code, const lead_decode_opts* opts, int32_t rounds, const uint32_t* syn,
                         int64_t shots, uint32_t* corr, uint8_t* status, int32_t* iters, float* llr,
                         void* workspace, size_t ws_bytes, void* stream);

/*
 * lead_osd -- ordered-statistics post-processing (OSD-CS) of the shots whose min-sum did not
 * converge (status without LEAD_ST_CONVERGED); the paper's global decoder is BP-OSD in the
 * osd_cs mode of order 3 (Sec. IV-A). Per such shot, on side opts->side:
 *  - qubits ordered by the BP posterior LLR post (ascending binary32 value through its
 *    order-preserving integer key, -0 before +0; ties by qubit index): most likely flipped first;
 *  - Gaussian elimination over GF(2) of H with its columns in that order and the syndrome
 *    carried along; the pivot of a column is the first remaining row with a 1 there; pivot
 *    columns form the basis S, the others T (same order);
 *  - candidates: OSD-0 (e_T = 0, e_S = H_S^-1 s), each single T column, each pair among the
 *    first `order` T columns (lexicographic); soft weight sum_{e_i = 1} W_i with
 *    W_i = rint(2^20 lambda_i), lambda the global decoder's binary32 prior LLRs, exact integer
 *    sums; ties to the earlier candidate;
 *  - corr[shot] is replaced by the chosen correction (it satisfies H e = s whenever s is in the
 *    column space of H, as for every syndrome of an error) and status[shot] gains LEAD_ST_OSD.
 *  order 0..6; codes with n and m[side] up to 65535 whose per-check elimination state (18 bytes
 *  per check of the side plus n/4 bytes) fits in one CTA's shared memory: m up to about 12 000.
 *  syn (dev, shots x words_m[side]); prior (dev, shots x n float, nullable: the channel LLR of
 *  opts->p for every qubit; for LEAD pass lead_local_estimate's output, the prior the global
 *  decoder used); post (dev, shots x n float): lead_decode's posterior LLRs; status (dev, in/out);
 *  corr (dev, in/out, shots x words_n).
 *  workspace (dev, 16-byte aligned) >= lead_osd_workspace_bytes: one m x ceil(n/64) x 8-byte
 *  matrix per CTA slot (at most two CTAs per SM) and, for codes whose sort and per-column arrays
 *  exceed shared memory, those arrays (about 8 np + 8 n + 8 m bytes, np the power of two >= n)
 *  per slot; a smaller workspace runs fewer slots.
 * Errors: LEAD_EINVAL, LEAD_ESTATE, LEAD_ECUDA.
 */
size_t lead_osd_workspace_bytes(const lead_code* code, const lead_decode_opts* opts, int64_t shots);
int lead_osd(const lead_code* code, const lead_decode_opts* opts, int32_t order, const uint32_t* syn, int64_t shots,
             const float* prior, const float* post, uint8_t* status, uint32_t* corr, void* workspace,
             size_t ws_bytes, void* stream);

/*
 * lead_check -- success test of Sec. IV-A on one side: residual r = err + corr.
 *  fail[shot] (dev uint8): bit 0 set iff H r != 0 (the correction misses the syndrome);
 *  bit 1 set iff H r = 0 and r is a nontrivial logical operator (it anticommutes with one of
 *  the code's logical operators of the other type, computed at build time by GF(2) elimination).
 *  err, corr (dev, shots x words_n).
 */
int lead_check(const lead_code* code, int32_t side, const uint32_t* err, const uint32_t* corr,
               int64_t shots, uint8_t* fail, void* stream);

/*
 * Continuous-batching decode server (the serving loop of the workload; the paper has no serving
 * layer). Requests are single shots of one of several codes prepared on the same device: both
 * sides' syndromes, an id and an arrival time. A dispatcher thread inside the library admits
 * each request once its arrival time has passed (times are nanoseconds on the server's clock,
 * lead_server_clock_ns), groups ready requests of one code into a batch of at most max_batch
 * shots whenever a stream slot is free, and keeps up to `streams` batches in flight (their
 * kernels overlap on the device). Each slot owns device buffers for max_batch shots; the number
 * of slots is min(streams, budget_bytes / slot size) (admission by memory; LEAD_EOOM if not even
 * one fits). Each batch runs the min-sum kernel in cfg->precision (as lead_decode with that
 * storage format; a 16-bit mode's kernel is compiled and loaded at creation), with the launch
 * shape lead_code_autotune kept nearest to the code's p_side, if any.
 * The two sides of a batch decode concurrently (two streams per slot).
 * lead_server_create builds, once, the Phase 1-2 tables of every code and side (the
 * local posterior table for the code's p and its class tables, as lead_decode would); every
 * batch then runs lead_decode's min-sum kernel on the sides in sides_mask with those tables and
 * copies corrections and statuses back; completion is detected with cudaEventQuery. A result
 * does not depend on the other requests of its batch (shots decode independently).
 */
typedef struct lead_server lead_server;

typedef struct {
  int32_t ncodes;
  lead_code* const* codes;   /* prepared on one device                                        */
  const double* p_side;      /* per code: channel marginal of each side (depolarizing p: 2p/3)  */
  int32_t sides_mask;        /* bit 0: decode side 0, bit 1: decode side 1                       */
  int32_t max_batch;         /* shots per launch                                                 */
  int32_t streams;           /* batches in flight                                                */
  size_t budget_bytes;       /* device memory the slots may use                                  */
  int32_t max_iter;
  float alpha;
  int32_t precision;         /* LEAD_PREC_*: storage format of the min-sum kernel (0 = binary32) */
} lead_server_config;

typedef struct {
  uint64_t id;
  int32_t code;
  uint8_t status[2];         /* LEAD_ST_* per side (0 for a side not decoded)                    */
  int64_t arrival_ns;        /* server clock                                                     */
  int64_t done_ns;           /* when the dispatcher saw the batch complete                       */
} lead_server_result;

int lead_server_create(const lead_server_config* cfg, lead_server** out);
/* n requests of code `code`: syn (host) rows of words_m[0] + words_m[1] words (side 0 then
 * side 1), ids (host), arrival_ns (host, nullable = now). Copies the data; returns at once. */
int lead_server_submit(lead_server* s, int32_t code, int64_t n, const uint32_t* syn, const uint64_t* ids,
                       const int64_t* arrival_ns);
/* Up to max completed results; corr (host, nullable) receives 2 x W words per result, W = the
 * largest words_n of the server's codes (side 0 row, then side 1 row). *got = results written. */
int lead_server_poll(lead_server* s, lead_server_result* out, uint32_t* corr, int64_t max, int64_t* got);
/* Requests submitted but not yet returned by lead_server_poll's queue (scheduled, ready, in flight). */
int lead_server_pending(lead_server* s, int64_t* pending);
int lead_server_clock_ns(lead_server* s, int64_t* t);
/* Stops the dispatcher, waits for the in-flight batches and frees the slots. */
void lead_server_destroy(lead_server* s);

/* Human-readable name of a status code (static string). */
const char* lead_status_string(int status);

/*
 * Checked build. The library built with LEAD_CHECKED (liblead_checked.so; the binding loads it
 * when LEAD_CHECKED=1 is set in the environment) has its kernels test every table-driven index
 * (partner slots, vertex and qubit ids, class ids, column positions) against its bound before
 * using it. A failed test skips the access and records the first failure on the device: site,
 * index and bound. lead_decode, lead_decode_noalloc, lead_local_estimate,
 * lead_local_estimate_priors, lead_decode_priors, lead_osd and lead_decode_iterated then wait
 * for their stream and return LEAD_ECHECK (a call captured into a CUDA graph does not wait; the
 * next eager call reports what the graph's replays recorded). The release build compiles the
 * tests out and never waits. This replaces a memory checker, which this build does not use.
 */
#define LEAD_BUILD_CHECKED 1
/*
 * lead_code_device_errors -- device error flags of a code's kernels (host, synchronous: waits
 * for the device). Bit 0 (LEAD_DEVERR_TC_WAIT): a per-qubit-prior kernel's wait for its
 * tensor-core operations ran out of its bound (the kernel stopped early and released its tensor
 * memory; the outputs of that call are incomplete). clear != 0 resets the flags.
 * Errors: LEAD_EINVAL, LEAD_ESTATE (not prepared, or another device current), LEAD_ECUDA.
 */
#define LEAD_DEVERR_TC_WAIT 1
int lead_code_device_errors(const lead_code* code, uint32_t* flags, int32_t clear);

/* LEAD_BUILD_* flags of the loaded library. */
int lead_build_flags(void);
/* The last failed check of a code, as {failures, site, index, bound}; all zero if none. */
int lead_code_check_record(const lead_code* code, uint64_t record[4]);

#ifdef __cplusplus
}
#endif
#endif /* LEAD_H */
