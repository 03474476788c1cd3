"""Exact local estimator of Phase 1 (Algorithm 1, Sec. III-B), oracle only.

Reading of the paper: LocalDecoder(H_v, s_v) returns the exact bitwise posterior under the
channel prior,

    q_{v,j} = P(e_j = 1 | H_v e = s_v) = sum_{e: H_v e = s_v} e_j pi(e) / sum_{e: H_v e = s_v} pi(e),

and the hard decision e_v = the coset member of least weight (the maximum-likelihood member
under a uniform prior p < 1/2), ties broken by the least row-major key
K(e) = sum_{a,b} E[a][b] 2^(a*Delta + b). The paper uses BP-LSD here and does not say which
soft vector it passes on; exact marginals are what LSD/OSD approximate.

With a uniform prior p, pi(e) = (1-p)^(n_l) r^wt(e) with r = p/(1-p), so

    q_{v,j} = N1_s,j(r) / N_s(r),   N_s(t) = sum_w N_s[w] t^w,  N1_s,j(t) = sum_w N1_s[j][w] t^w,

where N_s[w] counts the coset members of weight w and N1_s[j][w] those of them with e_j = 1.
These integer tables depend only on the local code, not on p.

How the tables are computed. Two exact integer identities for the defining sums are
implemented and must agree entry for entry:

* Fourier form (``fourier_tables``, the one ``tables`` uses): the indicator of H_v e = s is
  2^-m_l sum_u (-1)^(u.(H_v e + s)), and the weight-w sum of (-1)^(c.e) over e is the
  Krawtchouk value K_w(wt c), so N_s[w] = 2^-m_l sum_u (-1)^(u.s) K_w(wt(u H_v)).
* Row grouping (``row_tables``): the local check matrix is L = kron(R_B, R_A) (local index
  j = b*Delta + a), so for the Delta x Delta view E, L vec(E) = vec(R_A E R_B^T); writing
  f_a = R_B x_a for row a of E, the syndrome is S = R_A F with F the matrix of rows f_a, and
  the sum over E is a sum over the row images F with R_A F = S of the product over rows of
  P(f_a)(t) = sum_{x: R_B x = f_a} t^wt(x).

Further pins: brute force over all 2^(Delta^2) patterns for Delta = 4, the closed-form
marginals sum_s N_s[w] = C(n_l, w) and coset sizes 2^(n_l - m_l), MacWilliams on the zero
coset, and brute force over the coset for sampled syndromes at Delta = 6.
"""
from __future__ import annotations

import functools
from math import comb, factorial

import numpy as np


def _poly_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Row-wise product of integer polynomials: (N, da) x (N, db) -> (N, da+db-1)."""
    N, da = a.shape
    db = b.shape[1]
    out = np.zeros((N, da + db - 1), dtype=np.int64)
    for d in range(db):
        out[:, d:d + da] += a * b[:, d:d + 1]
    return out


def _row_tables(RB: np.ndarray):
    """For every row pattern x in F_2^Delta (bit b = x_b): f = R_B x as an integer (bit rB),
    its weight, and the per-(f) polynomials P(f)[w] and P_b(f)[w] (cached per R_B)."""
    RB = np.ascontiguousarray(RB, dtype=np.uint8)
    return _row_tables_cached(RB.tobytes(), RB.shape)


@functools.lru_cache(maxsize=16)
def _row_tables_cached(rb_bytes, rb_shape):
    RB = np.frombuffer(rb_bytes, dtype=np.uint8).reshape(rb_shape)
    kB, delta = RB.shape
    xs = np.arange(1 << delta)
    bits = (xs[:, None] >> np.arange(delta)[None, :]) & 1          # (2^Delta, Delta)
    f = ((bits @ RB.T.astype(np.int64)) & 1) @ (1 << np.arange(kB))
    wt = bits.sum(axis=1)
    P = np.zeros((1 << kB, delta + 1), dtype=np.int64)
    Pb = np.zeros((delta, 1 << kB, delta + 1), dtype=np.int64)
    for x in range(1 << delta):
        P[f[x], wt[x]] += 1
        for b in range(delta):
            if bits[x, b]:
                Pb[b, f[x], wt[x]] += 1
    return f, wt, bits, P, Pb


@functools.lru_cache(maxsize=16)
def _tables_cached(ra_bytes, ra_shape, rb_bytes, rb_shape):
    RA = np.frombuffer(ra_bytes, dtype=np.uint8).reshape(ra_shape)
    RB = np.frombuffer(rb_bytes, dtype=np.uint8).reshape(rb_shape)
    N, N1 = fourier_tables(np.kron(RB, RA).astype(np.uint8))
    return N, N1, ml_decisions(RA, RB)


def tables(RA: np.ndarray, RB: np.ndarray):
    """(N, N1, ml_mask): N (2^m_l, n_l+1), N1 (2^m_l, n_l, n_l+1) int64, ml_mask (2^m_l,) int64
    bit j = local index j of the ML hard decision. Cached per local code."""
    RA = np.ascontiguousarray(RA, dtype=np.uint8)
    RB = np.ascontiguousarray(RB, dtype=np.uint8)
    return _tables_cached(RA.tobytes(), RA.shape, RB.tobytes(), RB.shape)


def _row_images(RA: np.ndarray, RB: np.ndarray):
    """All row-image matrices F (f_a = (F >> a*kB) & mask) and their syndromes S = R_A F."""
    kA, delta = RA.shape
    kB = RB.shape[0]
    NF = 1 << (delta * kB)
    Fidx = np.arange(NF, dtype=np.int64)
    fa = np.stack([(Fidx >> (a * kB)) & ((1 << kB) - 1) for a in range(delta)])   # (Delta, NF)
    s_of_F = np.zeros(NF, dtype=np.int64)
    for rA in range(kA):
        for rB in range(kB):
            bit = np.zeros(NF, dtype=np.int64)
            for a in range(delta):
                if RA[rA, a]:
                    bit ^= (fa[a] >> rB) & 1
            s_of_F |= bit << (rB * kA + rA)
    return fa, s_of_F


def ml_decisions(RA: np.ndarray, RB: np.ndarray) -> np.ndarray:
    """ML hard decision per syndrome (least weight, then least row-major key), by grouping the
    coset by row images: for fixed F the members are products of independent row choices, so
    the best member takes in every row the least-weight, least-valued pattern x with R_B x = f_a;
    the best F minimises (total weight, key)."""
    kA, delta = RA.shape
    kB = RB.shape[0]
    m_l = kA * kB
    f_of_x, wt_of_x, _, _, _ = _row_tables(RB)
    fa, s_of_F = _row_images(RA, RB)
    minwt = np.full(1 << kB, 10 ** 9, dtype=np.int64)
    xmin = np.zeros(1 << kB, dtype=np.int64)
    for x in range(1 << delta):          # increasing x: first hit of the least weight is least x
        f = f_of_x[x]
        if wt_of_x[x] < minwt[f]:
            minwt[f] = wt_of_x[x]
            xmin[f] = x
    cost = sum(minwt[fa[a]] for a in range(delta))
    key = sum(xmin[fa[a]] << (a * delta) for a in range(delta))
    best_key = np.full(1 << m_l, -1, dtype=np.int64)
    srt = np.lexsort((key, cost))         # increasing (cost, key)
    s_sorted = s_of_F[srt]
    first = np.unique(s_sorted, return_index=True)[1]
    best_key[s_sorted[first]] = key[srt][first]
    ml_mask = np.zeros(1 << m_l, dtype=np.int64)
    for a in range(delta):
        for b in range(delta):
            bit = (best_key >> (a * delta + b)) & 1
            ml_mask |= bit << (b * delta + a)
    return ml_mask


def row_tables(RA: np.ndarray, RB: np.ndarray):
    """(N, N1) by grouping the defining sums by row images (see module doc)."""
    kA, delta = RA.shape
    kB = RB.shape[0]
    m_l = kA * kB
    n_l = delta * delta
    f_of_x, wt_of_x, _, P, Pb = _row_tables(RB)
    NF = 1 << (delta * kB)
    fa, s_of_F = _row_images(RA, RB)
    order = np.argsort(s_of_F, kind="stable")
    per = NF >> m_l
    if not (np.bincount(s_of_F, minlength=1 << m_l) == per).all():
        raise ValueError("local check matrix is not full rank")

    def group_sum(T):
        return T[order].reshape(1 << m_l, per, T.shape[1]).sum(axis=1)

    prod = P[fa[0]]
    for a in range(1, delta):
        prod = _poly_mul(prod, P[fa[a]])
    N = group_sum(prod)

    N1 = np.zeros((1 << m_l, n_l, n_l + 1), dtype=np.int64)
    # product over the other rows a2 != a, as (rows before a) * (rows after a)
    before = [np.ones((NF, 1), dtype=np.int64)]
    for a in range(delta - 1):
        before.append(_poly_mul(before[-1], P[fa[a]]))
    after = [np.ones((NF, 1), dtype=np.int64)]
    for a in range(delta - 1, 0, -1):
        after.append(_poly_mul(after[-1], P[fa[a]]))
    after = after[::-1]                    # after[a] = product over rows > a
    for a in range(delta):
        Q = _poly_mul(before[a], after[a])
        for b in range(delta):
            T = _poly_mul(Q, Pb[b][fa[a]])
            N1[:, b * delta + a, :] = group_sum(T)

    return N, N1


def posterior_from_tables(N: np.ndarray, N1: np.ndarray, p: float) -> np.ndarray:
    """q[s, j] in FP64: ratio of the two enumerator polynomials at r = p/(1-p), each evaluated
    by Horner's rule from the highest degree (separate IEEE multiply and add)."""
    if not (0.0 < p < 0.5):
        raise ValueError("the uniform prior must satisfy 0 < p < 1/2")
    r = p / (1.0 - p)
    deg = N.shape[-1] - 1
    num = np.zeros(N1.shape[:2], dtype=np.float64)
    den = np.zeros(N.shape[0], dtype=np.float64)
    for w in range(deg, -1, -1):
        num = num * r + N1[:, :, w].astype(np.float64)
        den = den * r + N[:, w].astype(np.float64)
    return num / den[:, None]


def brute_force(L: np.ndarray, delta: int):
    """(N, N1, ml_mask) by enumerating all 2^(Delta^2) local patterns (small Delta only)."""
    m_l, n_l = L.shape
    if n_l > 20:
        raise ValueError("brute force only for tiny local codes")
    es = np.arange(1 << n_l, dtype=np.int64)
    bits = ((es[:, None] >> np.arange(n_l)[None, :]) & 1).astype(np.int64)   # bit j = local j
    s = ((bits @ L.T.astype(np.int64)) & 1) @ (1 << np.arange(m_l))
    w = bits.sum(axis=1)
    N = np.zeros((1 << m_l, n_l + 1), dtype=np.int64)
    np.add.at(N, (s, w), 1)
    N1 = np.zeros((1 << m_l, n_l, n_l + 1), dtype=np.int64)
    for j in range(n_l):
        sel = bits[:, j] == 1
        np.add.at(N1[:, j, :], (s[sel], w[sel]), 1)
    # row-major key K(e) = sum E[a][b] 2^(a*Delta+b), local j = b*Delta + a
    key = np.zeros_like(es)
    for a in range(delta):
        for b in range(delta):
            key |= bits[:, b * delta + a] << (a * delta + b)
    ml = np.zeros(1 << m_l, dtype=np.int64)
    best = {}
    for idx in np.lexsort((key, w)):
        si = int(s[idx])
        if si not in best:
            best[si] = int(es[idx])
    for si, e in best.items():
        ml[si] = e
    return N, N1, ml


def posterior_brute_force(L: np.ndarray, s: int, p_vec: np.ndarray) -> np.ndarray:
    """The defining sum with an arbitrary per-position prior p_vec (small Delta only)."""
    m_l, n_l = L.shape
    es = np.arange(1 << n_l, dtype=np.int64)
    bits = ((es[:, None] >> np.arange(n_l)[None, :]) & 1)
    syn = ((bits @ L.T.astype(np.int64)) & 1) @ (1 << np.arange(m_l))
    sel = bits[syn == s].astype(np.float64)
    pi = np.prod(np.where(sel == 1, p_vec[None, :], 1.0 - p_vec[None, :]), axis=1)
    return (sel * pi[:, None]).sum(axis=0) / pi.sum()


def fourier_tables(L: np.ndarray):
    """(N, N1) from the Fourier form over the row space of L, in exact integers:
    N_s[w] = 2^-m_l sum_u (-1)^(u.s) K_w(wt(u L)), K_w(i) = sum_h (-1)^h C(i,h) C(n_l-i, w-h), and
    N1_s[j][w] = 2^-m_l sum_u (-1)^(u.s) (-1)^(c_j) K'_(w-1)(wt(c) - c_j) with c = u L and K'
    the Krawtchouk polynomial of length n_l - 1."""
    m_l, n_l = L.shape

    def kraw(length):
        K = np.zeros((length + 1, length + 1), dtype=object)   # K[w][i]
        for w in range(length + 1):
            for i in range(length + 1):
                K[w][i] = sum((-1) ** h * comb(i, h) * comb(length - i, w - h)
                              for h in range(0, min(i, w) + 1) if w - h <= length - i)
        return np.array(K.tolist(), dtype=np.int64)

    K = kraw(n_l)
    K1 = kraw(n_l - 1)
    us = np.arange(1 << m_l, dtype=np.int64)
    ubits = (us[:, None] >> np.arange(m_l)[None, :]) & 1
    C = (ubits @ L.astype(np.int64)) & 1                      # (2^m_l, n_l) codewords of rowspace
    wc = C.sum(axis=1)
    sgn = 1 - 2 * (np.bitwise_count((us[:, None] & us[None, :]).astype(np.uint64)) & 1).astype(np.int64)
    # sgn[u, s] = (-1)^(u.s)
    N = (sgn.T @ K[:, wc].T) >> m_l                            # (2^m_l, n_l+1)
    N1 = np.zeros((1 << m_l, n_l, n_l + 1), dtype=np.int64)
    for j in range(n_l):
        cj = C[:, j]
        col = np.zeros((1 << m_l, n_l + 1), dtype=np.int64)
        col[:, 1:] = ((1 - 2 * cj)[:, None] * K1[:, wc - cj].T)
        N1[:, j, :] = (sgn.T @ col) >> m_l
    return N, N1


def macwilliams_zero_coset(L: np.ndarray) -> np.ndarray:
    """Weight distribution of ker L from that of its dual (the row space of L) by MacWilliams:
    W_ker(x, y) = 2^-m_l sum_{c in rowspace L} (x + y)^(n_l - wt c) (x - y)^(wt c)."""
    m_l, n_l = L.shape
    us = np.arange(1 << m_l, dtype=np.int64)
    ubits = (us[:, None] >> np.arange(m_l)[None, :]) & 1
    wc = (((ubits @ L.astype(np.int64)) & 1).sum(axis=1))
    out = [0] * (n_l + 1)
    for i in wc.tolist():
        # coefficient of x^(n_l-w) y^w in (x+y)^(n_l-i) (x-y)^i
        for w in range(n_l + 1):
            out[w] += sum(comb(n_l - i, w - h) * comb(i, h) * (-1) ** h
                          for h in range(0, min(i, w) + 1) if w - h <= n_l - i)
    return np.array([x >> m_l for x in out], dtype=np.int64)


# ---------------------------------------------------------------------------------------
# Single-precision decision path. Floating point decides the hard decisions of the global
# decoder, so the oracle evaluates the prior LLR that feeds it in IEEE binary32 with a fixed
# operation order, as any single-precision implementation must:
#   * boost and merge in binary32, p clamped to [2^-23, 1 - 2^-23];
#   * lambda(p) = ln((1 - p)/p) is the binary32 rounding (to nearest, ties to even) of the exact
#     value: the plain definition. It is computed as 2 artanh(1 - 2p) in binary64 (an identity
#     for ln((1-p)/p); 1 - 2p is exact in binary64 for binary32 p), whose relative error is a few
#     2^-53; where that value lies so close to a binary32 rounding boundary that the error could
#     decide the rounding, the exact value is compared with the boundary in 60-digit decimal
#     arithmetic instead.
# ---------------------------------------------------------------------------------------

P_MIN_F = np.float32(2.0 ** -23)
P_MAX_F = np.float32(1.0 - 2.0 ** -23)


def _llr_exact_round(p: float) -> np.float32:
    """Binary32 rounding of ln((1-p)/p) for one binary32 p, decided in decimal arithmetic: the
    two binary32 neighbours of the binary64 estimate bracket the exact value, and the exact value
    is compared with their midpoint (p and every binary32 number are exact decimals)."""
    import decimal
    ctx = decimal.Context(prec=60)
    dp = decimal.Decimal(float(p))
    exact = ctx.ln(ctx.divide(ctx.subtract(decimal.Decimal(1), dp), dp))
    est = np.float32(float(exact))
    lo = np.nextafter(est, np.float32(-np.inf), dtype=np.float32)
    hi = np.nextafter(est, np.float32(np.inf), dtype=np.float32)
    best = est
    for cand in (lo, hi):          # the nearest of the three; ties to the even significand
        dc = abs(ctx.subtract(decimal.Decimal(float(cand)), exact))
        db = abs(ctx.subtract(decimal.Decimal(float(best)), exact))
        if dc < db or (dc == db and (int(np.float32(cand).view(np.uint32)) & 1) == 0):
            best = cand
    return np.float32(best)


def llr_f32(p: np.ndarray) -> np.ndarray:
    """lambda = ln((1 - p)/p) for binary32 p clamped to [2^-23, 1 - 2^-23], rounded to binary32
    (see the block comment above)."""
    p = np.clip(np.asarray(p, dtype=np.float32), P_MIN_F, P_MAX_F)
    y = 2.0 * np.arctanh(1.0 - 2.0 * p.astype(np.float64))
    lam = y.astype(np.float32)
    # distance of y from the rounding boundary next to lam, against 2^-49 |y| (well above the
    # binary64 error of artanh and of the doubling): only there can the rounding be in doubt
    al = np.abs(lam)
    a = al.astype(np.float64)
    half_up = (np.nextafter(al, np.float32(np.inf), dtype=np.float32).astype(np.float64) - a) / 2.0
    half_dn = (a - np.nextafter(al, np.float32(0), dtype=np.float32).astype(np.float64)) / 2.0
    d = np.abs(y - lam.astype(np.float64))
    tol = 2.0 ** -49 * np.abs(y)
    doubt = (np.abs(d - half_up) <= tol) | (np.abs(d - half_dn) <= tol)
    if doubt.any():
        flat_p, flat_l, flat_d = p.reshape(-1), lam.reshape(-1), doubt.reshape(-1)
        for k in np.nonzero(flat_d)[0]:
            flat_l[k] = _llr_exact_round(flat_p[k])
        lam = flat_l.reshape(p.shape)
    return lam.astype(np.float32)


# Cody-Waite split of ln 2 (the fdlibm pair): LN2_HI has its low 21 bits zero (32 significant
# bits), so k * LN2_HI is exact for |k| < 2^21, and LN2_HI + LN2_LO is ln 2 to double precision
# and beyond.
LN2_HI = np.array([0x3FE62E42FEE00000], dtype=np.uint64).view(np.float64)[0]
LN2_LO = np.array([0x3DEA39EF35793C76], dtype=np.uint64).view(np.float64)[0]
INV_LN2 = np.array([0x3FF71547652B82FE], dtype=np.uint64).view(np.float64)[0]   # nearest double to 1/ln 2


def exp_series_f64(x: np.ndarray) -> np.ndarray:
    """e^x for binary64 x in [-88, 88]: k = rint(x / ln 2), r = (x - k LN2_HI) - k LN2_LO
    (|r| <= ln 2 / 2 + tiny), e^r by its Taylor series through r^14 in Horner form (truncation
    below 1e-18), times 2^k (exact). Every step is a separate round-to-nearest binary64 operation."""
    x = np.asarray(x, dtype=np.float64)
    k = np.rint(x * INV_LN2)
    r = (x - k * LN2_HI) - k * LN2_LO
    s = np.full(x.shape, 1.0 / 87178291200.0)             # 1/14!
    for n in range(13, -1, -1):
        s = s * r
        s = s + 1.0 / float(factorial(n))
    return np.ldexp(s, k.astype(np.int64))


def sigmoid_f32(post: np.ndarray) -> np.ndarray:
    """q = 1 / (1 + e^post) as binary32: post (binary32) clamped to [-88, 88], then the binary64
    exponential above, add and divide, rounded once to binary32. (The probability that a qubit is
    flipped given its posterior LLR post = ln(P(0)/P(1)).)"""
    x = np.clip(np.asarray(post, dtype=np.float32), np.float32(-88.0), np.float32(88.0)).astype(np.float64)
    return (1.0 / (1.0 + exp_series_f64(x))).astype(np.float32)


# Binary32 constants of flip_prob_f32: 1/ln 2 and ln 2 = LN2_HI_F + LN2_LO_F with LN2_HI_F =
# 0.693359375 (9 significant bits, so k * LN2_HI_F is exact for |k| <= 25), each the binary64
# value rounded once to binary32; the Taylor coefficients 1/n! likewise.
INV_LN2_F = np.float32(1.4426950408889634)
LN2_HI_F = np.float32(0.693359375)
LN2_LO_F = np.float32(0.6931471805599453 - 0.693359375)
INV_FACT_F = [np.float32(1.0 / float(factorial(n))) for n in range(8)]
FLIP_CLAMP = np.float32(17.0)


def flip_prob_f32(post: np.ndarray) -> np.ndarray:
    """p = 1 / (1 + e^post), the flip probability a posterior LLR states, in binary32 arithmetic
    with every operation rounded to nearest: post clamped to [-17, 17] (beyond it p lies outside
    [2^-23, 1 - 2^-23], where the per-qubit prior is clamped anyway); k = rint(post / ln 2);
    r = (post - k LN2_HI_F) - k LN2_LO_F; e^r by its Taylor series through r^7 in Horner form;
    e^post = e^r 2^k (exact); then the add and the divide."""
    x = np.clip(np.asarray(post, dtype=np.float32), -FLIP_CLAMP, FLIP_CLAMP).astype(np.float32)
    k = np.rint((x * INV_LN2_F).astype(np.float32)).astype(np.float32)
    r = ((x - (k * LN2_HI_F).astype(np.float32)).astype(np.float32) - (k * LN2_LO_F).astype(np.float32))
    r = r.astype(np.float32)
    s = np.full(x.shape, INV_FACT_F[7], dtype=np.float32)
    for n in range(6, -1, -1):
        s = ((s * r).astype(np.float32) + INV_FACT_F[n]).astype(np.float32)
    e = np.ldexp(s, k.astype(np.int32)).astype(np.float32)
    return (np.float32(1.0) / (np.float32(1.0) + e).astype(np.float32)).astype(np.float32)


def boosted_table_f32(N, N1, ml_mask, p: float) -> np.ndarray:
    """Phase-1 output table in binary32: q rounded to binary32, then max(q, 1/2) on the bits of
    the ML decision (the boost of Algorithm 1; the ML member always satisfies H_v e = s_v)."""
    q = posterior_from_tables(N, N1, p).astype(np.float32)
    n_l = q.shape[1]
    flip = ((ml_mask[:, None] >> np.arange(n_l)[None, :]) & 1).astype(bool)
    return np.where(flip, np.maximum(q, np.float32(0.5)), q).astype(np.float32)


# ---------------------------------------------------------------------------------------
# Per-qubit (non-uniform) priors. The defining sums are the same, with pi(e) the product of the
# qubits' own Bernoulli priors p_j. They are evaluated by the row grouping of the module doc in
# FP64, with row weights relative to the all-zero row: r_a(x) = prod_{b: x_b = 1} p_ab/(1 - p_ab).
# The hard decision is the ML member, the least cost sum_j e_j W_j with integer costs
# W_j = rint(2^20 * lambda_f32(p_j)) (exact sums, so uniform priors reproduce the integer-weight
# decision), ties broken by the least row-major key as in the uniform case.
# ---------------------------------------------------------------------------------------

@functools.lru_cache(maxsize=16)
def _cosets_cached(ra_bytes, ra_shape, rb_bytes, rb_shape):
    """The row-image matrices grouped by syndrome: (fa sorted by S = R_A F, start of each S)."""
    RA = np.frombuffer(ra_bytes, dtype=np.uint8).reshape(ra_shape)
    RB = np.frombuffer(rb_bytes, dtype=np.uint8).reshape(rb_shape)
    fa, s_of_F = _row_images(RA, RB)
    order = np.argsort(s_of_F, kind="stable")
    starts = np.searchsorted(s_of_F[order], np.arange((1 << (ra_shape[0] * rb_shape[0])) + 1))
    return fa[:, order], starts


def coset_row_images(RA: np.ndarray, RB: np.ndarray, s: int):
    """All row-image matrices F (as (Delta,) arrays of f_a) with R_A F = S, for syndrome s, in
    increasing order of their packed value (the shot-invariant grouping is cached per local code)."""
    RA = np.ascontiguousarray(RA, dtype=np.uint8)
    RB = np.ascontiguousarray(RB, dtype=np.uint8)
    fa, starts = _cosets_cached(RA.tobytes(), RA.shape, RB.tobytes(), RB.shape)
    return fa[:, starts[s]:starts[s + 1]]


def posterior_nonuniform(RA: np.ndarray, RB: np.ndarray, s: int, p: np.ndarray) -> np.ndarray:
    """q_j = P(e_j = 1 | H_v e = s) for per-position priors p (local index j = b*Delta + a), FP64."""
    kA, delta = RA.shape
    f_of_x, _, bits, _, _ = _row_tables(RB)
    kB = RB.shape[0]
    P = np.asarray(p, dtype=np.float64).reshape(delta, delta).T            # P[a][b] = p_{b*Delta + a}
    odds = P / (1.0 - P)
    R = np.zeros((delta, 1 << kB))
    Rb = np.zeros((delta, delta, 1 << kB))
    for a in range(delta):
        w = np.prod(np.where(bits == 1, odds[a][None, :], 1.0), axis=1)      # r_a(x), x = 0..2^Delta-1
        np.add.at(R[a], f_of_x, w)
        for b in range(delta):
            sel = bits[:, b] == 1
            np.add.at(Rb[a, b], f_of_x[sel], w[sel])
    F = coset_row_images(RA, RB, s)                                        # (Delta, #F)
    terms = np.prod(np.stack([R[a][F[a]] for a in range(delta)]), axis=0)  # prod_a R_a(f_a)
    Z = terms.sum()
    q = np.zeros((delta, delta))
    for a in range(delta):
        others = terms / R[a][F[a]]
        for b in range(delta):
            q[a, b] = (others * Rb[a, b][F[a]]).sum() / Z
    return q.T.reshape(-1)                                                 # back to j = b*Delta + a


def integer_costs(p: np.ndarray) -> np.ndarray:
    """W_j = rint(2^20 * lambda_f32(p_j)) as int64 (binary32 lambda, exact scaling, round half even)."""
    lam = llr_f32(np.asarray(p, dtype=np.float32))
    return np.rint((lam * np.float32(2 ** 20)).astype(np.float32)).astype(np.int64)


def ml_nonuniform(RA: np.ndarray, RB: np.ndarray, s: int, W: np.ndarray) -> int:
    """Least (sum_j e_j W_j, row-major key) coset member for integer costs W (local order j)."""
    kA, delta = RA.shape
    f_of_x, _, bits, _, _ = _row_tables(RB)
    Wm = np.asarray(W, dtype=np.int64).reshape(delta, delta).T            # Wm[a][b]
    F = coset_row_images(RA, RB, s)
    kB = RB.shape[0]
    best_row = np.zeros((delta, 1 << kB, 2), dtype=np.int64)               # (cost, least x) per class
    for a in range(delta):
        cost = bits @ Wm[a]
        for f in range(1 << kB):
            xs = np.nonzero(f_of_x == f)[0]
            c = cost[xs]
            m = c.min()
            best_row[a, f] = (m, xs[c == m].min())
    tot = sum(best_row[a, F[a], 0] for a in range(delta))
    key = sum(best_row[a, F[a], 1] << (a * delta) for a in range(delta))
    i = np.lexsort((key, tot))[0]
    mask = 0
    for a in range(delta):
        x = int(best_row[a, F[a, i], 1])
        for b in range(delta):
            if (x >> b) & 1:
                mask |= 1 << (b * delta + a)
    return mask
