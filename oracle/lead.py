"""Algorithm 1 (LEAD decoder) and the failure criterion of Sec. IV-A; oracle only.

One decoding side at a time (Sec. III focuses on one error type; the other follows by
symmetry): side 0 takes the H_Z syndrome of X errors and the V0 local views, side 1 the H_X
syndrome of Z errors and the V1 local views. Depolarizing noise decodes both sides, each with
the marginal prior 2p/3 of its error type.

Phase 1 (local decoding + boost): s_v is the contiguous m_l-bit field of the syndrome at
vertex v (checks v*m_l .. v*m_l + m_l - 1); the exact local estimator of ``local`` gives q_v
and the ML decision e_v, which always satisfies H_v e_v = s_v, so the boost
q_{v,j} <- max(q_{v,j}, 1/2) applies to every bit with e_{v,j} = 1.
Phase 2 (regularisation): every qubit lies in exactly two views of a side (|S_i| = 2 under TNC),
p_i = alpha * (q_{v0,j0} + q_{v1,j1}) / 2.  The prior LLR is ln((1 - p_i)/p_i) with p_i clamped
to [2^-23, 1 - 2^-23] (the paper does not state a clamp; this one keeps binary32 finite).
Phase 3 (global decoder): flooding min-sum with scaling 1 and at most ``max_iter`` iterations
(the BP part of the paper's BP-OSD global decoder; OSD-CS post-processing is in ``osd``).

Two numeric tracks:
* ``prior_f64``: q, p_i and the LLR in FP64 -- the quantities the single-precision path must
  reproduce within its tolerance; ``decode_f64`` continues it with min-sum in FP64 (same rules
  and order), the reference for how often binary32 rounding changes a decision;
* the decision track in IEEE binary32 (``prior_f32`` and ``min_sum``), because floating point
  decides the hard decisions: q rounded to binary32, the boost and merge in binary32, the LLR
  by ``local.llr_f32``; min-sum messages in binary32 with this fixed order of additions:
  post_i = (lambda_i + U_{v0,j0}) + U_{v1,j1}, v0 < v1 the two views of qubit i, and
  U_{v,j} = sum over the local rows r containing j, in increasing r, of the check-to-qubit
  messages, accumulated from 0.  v2c = post - c2v; c2v = (-1)^(s_c + number of negative other
  v2c) * min over the other |v2c|.  The hard decision is e_i = [post_i < 0].
  Iteration 0 checks the prior's own hard decision; iteration t >= 1 checks after the t-th
  message update; the first t with H e = s stops (status bit 0); otherwise status bit 1 and the
  last decision is returned.

Storage precision (a serving extension; the paper uses one precision): in the bfloat16 and
binary16 modes every LLR the decoder keeps between steps is rounded to nearest even into that
format when stored -- the prior lambda_i, the check-to-qubit magnitudes (the sign is applied
after rounding), each per-view sum U_{v,j} (accumulated in binary32, rounded once), and the
posterior post_i; arithmetic stays binary32 and the hard decision reads the stored posterior.
Binary16 storage saturates at +-65504 (min-sum magnitudes can outgrow its range over many
iterations; an infinity would turn later differences into NaN). The sign of a v2c message is
its IEEE sign bit (a zero difference is +0 in binary32, but a
binary16 posterior can underflow to -0).

Parity: phases 1-2 are pinned through ``local``; the merge by the Appendix-A worked example;
min-sum by its textbook special cases (exact ML on a cycle-free check matrix, zero syndrome
-> zero correction at iteration 0, every converged output satisfies H e = s). Beyond those,
min-sum parity is "parity unpinned" except against the single-precision implementation.
"""
from __future__ import annotations

import numpy as np

from . import gf2, local
from .tanner import TannerCode

STATUS_CONVERGED = 1
STATUS_MAX_ITER = 2
PREC_FP32, PREC_BF16, PREC_FP16 = 0, 1, 2
EST_EXACT, EST_MINSUM = 0, 1      # local decoders of Phase 1


def round_bf16(x: np.ndarray) -> np.ndarray:
    """binary32 -> nearest bfloat16 (ties to even) -> binary32: keep the top 16 bits of the
    binary32 pattern after adding half an ulp of the kept part (plus one when the kept part is
    odd). Finite inputs."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def round_storage(x: np.ndarray, precision: int) -> np.ndarray:
    """The stored value of binary32 x in a precision mode, as binary32."""
    x = np.asarray(x, dtype=np.float32)
    if precision == PREC_FP32:
        return x
    if precision == PREC_BF16:
        return round_bf16(x)
    if precision == PREC_FP16:       # saturating at the largest finite binary16
        return np.clip(x, np.float32(-65504.0), np.float32(65504.0)).astype(np.float16).astype(np.float32)
    raise ValueError(precision)


def local_syndromes(side: Side, syn: np.ndarray) -> np.ndarray:
    """s_v as integers (bit r = syndrome bit v*m_l + r) for syn (S, m) 0/1 -> (S, |G|)."""
    S, m = syn.shape
    m_l = side.m_l
    fields = syn.reshape(S, m // m_l, m_l).astype(np.int64)
    return (fields << np.arange(m_l)[None, None, :]).sum(axis=2)


def merge_f64(q0: np.ndarray, q1: np.ndarray, alpha: float) -> np.ndarray:
    """Phase 2: p_i = alpha * Average(S_i) with |S_i| = 2."""
    return alpha * (q0 + q1) / 2.0


def prior_f64(code: TannerCode, side_id: int, syn: np.ndarray, p: float, alpha: float = 1.0):
    """Phases 1-2 in FP64: returns (p_hat (S, n), llr (S, n))."""
    side = code.sides[side_id]
    N, N1, ml = local.tables(side.RA, side.RB)
    q = local.posterior_from_tables(N, N1, p)                         # (2^m_l, n_l)
    n_l = q.shape[1]
    flip = ((ml[:, None] >> np.arange(n_l)[None, :]) & 1).astype(bool)
    qb = np.where(flip, np.maximum(q, 0.5), q)                        # boost
    sv = local_syndromes(side, syn)                                   # (S, |G|)
    qv = side.qubit_views
    q0 = qb[sv[:, qv[:, 0, 0]], qv[:, 0, 1]]
    q1 = qb[sv[:, qv[:, 1, 0]], qv[:, 1, 1]]
    ph = merge_f64(q0, q1, alpha)
    pc = np.clip(ph, 2.0 ** -23, 1.0 - 2.0 ** -23)
    return ph, np.log((1.0 - pc) / pc)


def prior_f32(code: TannerCode, side_id: int, syn: np.ndarray, p: float, alpha: float = 1.0,
              estimator: int = EST_EXACT):
    """Phases 1-2 on the binary32 decision track: returns llr (S, n) float32. estimator selects
    the local decoder: the exact posterior (EST_EXACT) or local min-sum BP (EST_MINSUM)."""
    side = code.sides[side_id]
    if estimator == EST_MINSUM:
        lut = local_minsum_tables(side.RA, side.RB, p)[0]
    else:
        N, N1, ml = local.tables(side.RA, side.RB)
        lut = local.boosted_table_f32(N, N1, ml, p)
    sv = local_syndromes(side, syn)
    qv = side.qubit_views
    q0 = lut[sv[:, qv[:, 0, 0]], qv[:, 0, 1]]
    q1 = lut[sv[:, qv[:, 1, 0]], qv[:, 1, 1]]
    h = (q0 + q1).astype(np.float32)
    h = (h * np.float32(0.5)).astype(np.float32)
    ph = (h * np.float32(alpha)).astype(np.float32)
    return local.llr_f32(ph)


def channel_prior_f32(n: int, shots: int, p: float) -> np.ndarray:
    """The standalone BP baseline's prior: the channel LLR of p for every qubit (binary32)."""
    return np.broadcast_to(local.llr_f32(np.array([p], dtype=np.float32)), (shots, n)).copy()


def local_priors(code: TannerCode, side_id: int, syn: np.ndarray, prior: np.ndarray, boost: bool = True):
    """Phase 1 with per-qubit priors: local posteriors q (S, |G|, n_l) in FP64, boosted to 1/2 on
    the bits of the least-cost local decision unless boost=False, and those decisions (S, |G|) as
    masks (bit j = local index j). prior (S, n)."""
    side = code.sides[side_id]
    sv = local_syndromes(side, syn)
    S, V = sv.shape
    nl = side.views.shape[1]
    q = np.zeros((S, V, nl))
    ml = np.zeros((S, V), dtype=np.int64)
    for s in range(S):
        for v in range(V):
            pv = prior[s, side.views[v]]
            qq = local.posterior_nonuniform(side.RA, side.RB, int(sv[s, v]), pv.astype(np.float64))
            m = local.ml_nonuniform(side.RA, side.RB, int(sv[s, v]), local.integer_costs(pv))
            flip = ((m >> np.arange(nl)) & 1).astype(bool)
            q[s, v] = np.where(flip, np.maximum(qq, 0.5), qq) if boost else qq
            ml[s, v] = m
    return q, ml


def merge_priors_f32(code: TannerCode, side_id: int, q: np.ndarray, alpha: float = 1.0) -> np.ndarray:
    """Phase 2 on per-view boosted posteriors q (S, |G|, n_l), binary32 decision track:
    lambda(alpha * ((q0 + q1) * 1/2)) per qubit, q rounded to binary32 first."""
    qv = code.sides[side_id].qubit_views
    q32 = q.astype(np.float32)
    q0 = q32[:, qv[:, 0, 0], qv[:, 0, 1]]
    q1 = q32[:, qv[:, 1, 0], qv[:, 1, 1]]
    h = (q0 + q1).astype(np.float32)
    h = (h * np.float32(0.5)).astype(np.float32)
    return local.llr_f32((h * np.float32(alpha)).astype(np.float32))


class _Graph:
    """Edge lists of a check matrix whose rows come in consecutive blocks of ``block`` rows
    (the checks of one vertex). For every qubit, its edges are grouped by block in increasing
    block order and, inside a block, in increasing row order."""

    def __init__(self, H: np.ndarray, block: int):
        H = np.asarray(H, dtype=np.uint8)
        self.H = H
        self.m, self.n = H.shape
        rows = [np.nonzero(H[c])[0] for c in range(self.m)]
        dmax = max(1, max(len(x) for x in rows))
        self.nbr = np.zeros((self.m, dmax), dtype=np.int64)
        self.valid = np.zeros((self.m, dmax), dtype=bool)
        for c, js in enumerate(rows):
            self.nbr[c, :len(js)] = js
            self.valid[c, :len(js)] = True
        per_qubit = [dict() for _ in range(self.n)]
        for c, js in enumerate(rows):
            for k, i in enumerate(js):
                per_qubit[i].setdefault(c // block, []).append(c * dmax + k)
        nb = max(1, max(len(d) for d in per_qubit))
        nu = max(1, max((len(v) for d in per_qubit for v in d.values()), default=1))
        # edge[i, t, u] = flat edge id of the u-th check of the t-th block of qubit i, or -1
        self.edge = -np.ones((self.n, nb, nu), dtype=np.int64)
        for i, d in enumerate(per_qubit):
            for t, b in enumerate(sorted(d)):
                for u, eid in enumerate(d[b]):
                    self.edge[i, t, u] = eid


def _syndrome_of(H: np.ndarray, e: np.ndarray) -> np.ndarray:
    """H e mod 2 per row of e (float64 products are exact integers here)."""
    return (np.rint(e.astype(np.float64) @ H.T.astype(np.float64)).astype(np.int64) & 1).astype(np.uint8)


def min_sum(H: np.ndarray, block: int, syn: np.ndarray, llr: np.ndarray, max_iter: int = 32,
            early_stop: bool = True, precision: int = PREC_FP32, dtype=np.float32):
    """Phase 3, flooding min-sum in binary32 on the check matrix H whose rows come in blocks of
    ``block`` (one block per vertex view; the order of additions is documented in the module
    doc). syn (S, m) 0/1, llr (S, n) float32 -> (corr (S, n) uint8, status (S,) uint8,
    iters (S,) int32, post (S, n) float32 final posterior LLRs).
    ``early_stop=False`` runs all ``max_iter`` iterations and reports the last decision (used to
    pin the message rules against the fixed point on cycle-free graphs). ``precision`` selects
    the storage format of the module doc. ``dtype=np.float64`` runs the same rules and order in
    binary64 (the FP64 reference track; posteriors are then returned in binary64)."""
    ft = np.dtype(dtype).type
    if ft is np.float64 and precision != PREC_FP32:
        raise ValueError("storage modes are defined on the binary32 track")
    R = lambda x: round_storage(x, precision)  # noqa: E731
    g = _Graph(H, block)
    S, n = llr.shape
    lam = R(llr.astype(ft))
    corr = np.zeros((S, n), dtype=np.uint8)
    status = np.zeros(S, dtype=np.uint8)
    iters = np.zeros(S, dtype=np.int32)
    post_out = np.zeros((S, n), dtype=ft)
    active = np.arange(S)
    dmax = g.nbr.shape[1]
    c2v = np.zeros((S, g.m, dmax), dtype=ft)
    post = lam.copy()
    sgn_s = syn.astype(bool)
    edge_ok = g.edge >= 0
    edge_ix = np.where(edge_ok, g.edge, 0)
    for t in range(0, max_iter + 1):
        if t > 0:
            # check-node update for the active shots
            pa = post[active]
            v2c = (pa[:, g.nbr] - c2v[active]).astype(ft)
            mag = np.where(g.valid[None], np.abs(v2c), ft(np.inf)).astype(ft)
            neg = np.signbit(v2c) & g.valid[None]
            # min over the other slots of a check = min(prefix minimum before k, suffix after k)
            inf = np.full(mag.shape[:2] + (1,), np.inf, dtype=ft)
            pre = np.concatenate([inf, np.minimum.accumulate(mag, axis=2)[:, :, :-1]], axis=2)
            suf = np.concatenate([np.minimum.accumulate(mag[:, :, ::-1], axis=2)[:, :, ::-1][:, :, 1:],
                                  inf], axis=2)
            mn = R(np.minimum(pre, suf))
            # parity of the other slots' signs = parity of all of them XOR the slot's own sign
            par = ((neg.sum(axis=2) & 1).astype(bool)[:, :, None] ^ neg) ^ sgn_s[active][:, :, None]
            new = np.where(par, -mn, mn).astype(ft)
            new = np.where(g.valid[None], new, ft(0.0)).astype(ft)
            c2v[active] = new
            # variable-node update: per-block sums in increasing row, blocks in increasing order
            flat = new.reshape(new.shape[0], -1)
            acc = lam[active].copy()
            for tb in range(g.edge.shape[1]):
                U = np.zeros((active.size, n), dtype=ft)
                for u in range(g.edge.shape[2]):
                    ok = edge_ok[:, tb, u]
                    vals = np.where(ok[None], flat[:, edge_ix[:, tb, u]], ft(0.0))
                    U = (U + vals).astype(ft)
                has = edge_ok[:, tb, 0]
                acc = np.where(has[None], (acc + R(U)).astype(ft), acc).astype(ft)
            post[active] = R(acc)
        e = (post[active] < 0).astype(np.uint8)
        ok = (_syndrome_of(g.H, e) == syn[active]).all(axis=1)
        if not early_stop and t < max_iter:
            ok[:] = False
        done = active[ok]
        corr[done] = e[ok]
        status[done] = STATUS_CONVERGED
        iters[done] = t
        post_out[done] = post[done]
        if t == max_iter:
            rest = active[~ok]
            corr[rest] = e[~ok]
            status[rest] = STATUS_MAX_ITER
            iters[rest] = max_iter
            post_out[rest] = post[rest]
        active = active[~ok]
        if active.size == 0:
            break
    return corr, status, iters, post_out


def decode(code: TannerCode, side_id: int, syn: np.ndarray, p: float, alpha: float = 1.0,
           max_iter: int = 32, use_lead: bool = True, precision: int = PREC_FP32,
           estimator: int = EST_EXACT):
    """Algorithm 1 on one side (use_lead=False: the standalone min-sum baseline)."""
    if use_lead:
        lam = prior_f32(code, side_id, syn, p, alpha, estimator)
    else:
        lam = channel_prior_f32(code.n, syn.shape[0], p)
    side = code.sides[side_id]
    return min_sum(side.H, side.m_l, syn, lam, max_iter, precision=precision)


def decode_f64(code: TannerCode, side_id: int, syn: np.ndarray, p: float, alpha: float = 1.0,
               max_iter: int = 32, use_lead: bool = True):
    """Algorithm 1 on the FP64 track: the prior LLRs of ``prior_f64`` (or the channel LLR
    ln((1-p)/p) in binary64 for use_lead=False) and min-sum in binary64 with the same rules and
    order. It measures how often the binary32 decision track decides differently."""
    if use_lead:
        _, lam = prior_f64(code, side_id, syn, p, alpha)
    else:
        lam = np.full((syn.shape[0], code.n), np.log((1.0 - p) / p))
    side = code.sides[side_id]
    return min_sum(side.H, side.m_l, syn, lam, max_iter, dtype=np.float64)


def redecode(code: TannerCode, side_id: int, syn: np.ndarray, post: np.ndarray, alpha: float = 1.0,
             max_iter: int = 32, use_lead: bool = True, precision: int = PREC_FP32):
    """One round of iterated LEAD (an extension; the paper runs Algorithm 1 once): the per-qubit
    prior is the flip probability the last global posterior LLR states, p_i = 1 / (1 + e^{post_i})
    (``local.flip_prob_f32``, binary32), clamped to [2^-23, 1 - 2^-23]; then Algorithm 1 with that prior:
    Phase 1 the exact local posterior under the product prior with its least-cost decision and
    boost (``local_priors``), Phase 2 ``merge_priors_f32``, Phase 3 ``min_sum``. use_lead=False
    hands lambda(p_i) to min-sum directly. Returns (corr, status, iters, post) as ``decode``."""
    prior = np.clip(local.flip_prob_f32(post), local.P_MIN_F, local.P_MAX_F).astype(np.float32)
    if use_lead:
        q, _ = local_priors(code, side_id, syn, prior)
        lam = merge_priors_f32(code, side_id, q, alpha)
    else:
        lam = local.llr_f32(prior)
    side = code.sides[side_id]
    return min_sum(side.H, side.m_l, syn, lam, max_iter, precision=precision)


def decode_iterated(code: TannerCode, side_id: int, syn: np.ndarray, p: float, rounds: int, alpha: float = 1.0,
                    max_iter: int = 32, use_lead: bool = True, precision: int = PREC_FP32,
                    estimator: int = EST_EXACT):
    """Iterated LEAD: round 0 is ``decode``; each further round applies ``redecode`` to the shots
    whose status lacks STATUS_CONVERGED, with their last posteriors. Converged shots keep their
    round's result, and iterations add up over the rounds a shot ran. Returns (corr, status,
    iters, post) as ``decode``."""
    corr, st, it, post = decode(code, side_id, syn, p, alpha, max_iter, use_lead, precision, estimator)
    for _ in range(1, rounds):
        sel = np.nonzero((st & STATUS_CONVERGED) == 0)[0]
        if sel.size == 0:
            break
        c, s, i, pst = redecode(code, side_id, syn[sel], post[sel], alpha, max_iter, use_lead, precision)
        corr[sel] = c
        st[sel] = s
        it[sel] += i
        post[sel] = pst
    return corr, st, it, post


def check(code: TannerCode, side_id: int, err: np.ndarray, corr: np.ndarray) -> np.ndarray:
    """Sec. IV-A success test on one side: residual r = e + e_hat. bit 0: H r != 0 (the
    estimate does not reproduce the syndrome); bit 1: H r = 0 but r is not a stabilizer
    (r outside the row space of the other side's check matrix), a logical error."""
    H = code.sides[side_id].H
    other = code.sides[1 - side_id].H
    r = (err ^ corr).astype(np.uint8)
    bad_syn = _syndrome_of(H, r).any(axis=1)
    R, piv = gf2.rref(other)
    x = r.copy()
    for i, c in enumerate(piv):
        hit = x[:, c] == 1
        if hit.any():
            x[hit] ^= R[i]
    logical = x.any(axis=1) & ~bad_syn
    return (bad_syn.astype(np.uint8) | (logical.astype(np.uint8) << 1)).astype(np.uint8)


def local_minsum_tables(RA: np.ndarray, RB: np.ndarray, p: float, max_iter: int | None = None):
    """Phase 1 with local min-sum BP as the LocalDecoder (the paper's local decoders are BP based,
    with at most as many iterations as the local code length, Sec. IV-A): for every local
    syndrome s, flooding min-sum on the local check matrix kron(R_B, R_A) with the binary32
    channel LLR lambda_f32(p) on every position, exactly the global rules of ``min_sum`` (one
    vertex block), at most Delta^2 iterations. The soft output is q_j = sigmoid_f32(post_j); when
    the hard decision satisfies the local syndrome, q_j <- max(q_j, 1/2) on its flipped bits
    (Alg. 1 Phase 1). A uniform prior makes the result a function of s alone, so it is a table.
    Returns (table (2^m_l, n_l) float32, iterations (2^m_l,) int32, converged (2^m_l,) bool,
    hard decisions (2^m_l, n_l) uint8)."""
    RA = np.asarray(RA, dtype=np.uint8)
    RB = np.asarray(RB, dtype=np.uint8)
    H = np.kron(RB, RA).astype(np.uint8)                 # local row r = rB * kA + rA
    m_l, n_l = H.shape
    S = 1 << m_l
    syn = ((np.arange(S)[:, None] >> np.arange(m_l)[None, :]) & 1).astype(np.uint8)
    lam = np.broadcast_to(local.llr_f32(np.array([p], dtype=np.float32)), (S, n_l)).copy()
    corr, status, iters, post = min_sum(H, m_l, syn, lam, n_l if max_iter is None else max_iter)
    q = local.sigmoid_f32(post)
    conv = status == STATUS_CONVERGED
    boost = conv[:, None] & (corr == 1)
    q = np.where(boost, np.maximum(q, np.float32(0.5)), q).astype(np.float32)
    return q, iters.astype(np.int32), conv, corr


def expected_local_iterations(RA: np.ndarray, RB: np.ndarray, p: float, iters: np.ndarray) -> float:
    """E[I_l] per vertex under i.i.d. flips with probability p: sum_s P(s) I_l(s), with P(s) from
    the coset weight enumerators, P(s) = sum_w N_s[w] p^w (1 - p)^(n_l - w)."""
    N, _, _ = local.tables(RA, RB)
    n_l = N.shape[1] - 1
    w = np.arange(n_l + 1)
    ps = (N.astype(np.float64) * (p ** w) * ((1.0 - p) ** (n_l - w))).sum(axis=1)
    return float((ps * np.asarray(iters, dtype=np.float64)).sum())

