"""Ordered-statistics decoding (OSD) after min-sum; oracle only (test infrastructure).

The paper's global decoder is BP-OSD in the `osd_cs` mode of order 3 (Sec. IV-A): when BP does
not produce a correction that satisfies the syndrome, OSD does. This module writes that step out
for one side's check matrix H (m x n), per shot:

1. Order the qubits by the BP posterior LLR, most likely flipped first: ascending posterior,
   with binary32 values compared through their order-preserving integer key (-0 before +0), and
   ties broken by the qubit index.
2. Gaussian elimination over GF(2) of H with its columns in that order, the syndrome carried
   along as an extra column. For each column in turn, the pivot is the first remaining row
   (current row order) with a 1 in that column. It is swapped into the next pivot position and
   added to every other row with a 1 there. Pivot columns form the basis S; the others, in the
   same order, form T.
3. Candidates (order lam):
   - OSD-0, with e_T = 0 and e_S = H_S^-1 s;
   - every single flip of a T column;
   - every pair among the first lam T columns, pairs in lexicographic order.
   For a flip set C of T columns, e_T = 1_C and e_S = H_S^-1 (s + H_C 1).
4. Ranking by soft weight sum_{i: e_i = 1} W_i. Here W_i = rint(2^20 lambda_i), with lambda the
   binary32 prior LLRs that the global decoder was given: the channel model the decoder trusts.
   Sums are exact integers, and ties go to the earlier candidate in the order above.

Every candidate satisfies H e = s whenever s lies in the column space of H. This holds for
syndromes of actual errors.
"""
from __future__ import annotations

import numpy as np


def order_keys(post: np.ndarray) -> np.ndarray:
    """Order-preserving uint32 keys of binary32 values (negative values reversed)."""
    u = np.ascontiguousarray(post, dtype=np.float32).view(np.uint32).astype(np.uint64)
    neg = (u >> 31) == 1
    return np.where(neg, (~u) & 0xFFFFFFFF, u | 0x80000000).astype(np.uint64)


def column_order(post: np.ndarray) -> np.ndarray:
    """Qubit indices, most likely flipped first (ascending posterior LLR, ties by index)."""
    n = post.shape[0]
    return np.lexsort((np.arange(n), order_keys(post)))


def integer_weights(prior: np.ndarray) -> np.ndarray:
    """W_i = rint(2^20 lambda_i) (binary32 product, exact scaling, round half to even)."""
    lam = np.asarray(prior, dtype=np.float32)
    return np.rint((lam * np.float32(2 ** 20)).astype(np.float32)).astype(np.int64)


def eliminate(H: np.ndarray, s: np.ndarray, order: np.ndarray):
    """Row reduction of H[:, order] with the syndrome as an extra column. Returns (M (rows,
    n) uint8 reduced matrix in column-order coordinates, s' (rows,), pivot columns (list of
    positions in column order), rank)."""
    M = np.ascontiguousarray(H[:, order], dtype=np.uint8).copy()
    sv = np.asarray(s, dtype=np.uint8).copy()
    m, n = M.shape
    rank = 0
    pivots = []
    for col in range(n):
        if rank == m:
            break
        rows = np.nonzero(M[rank:, col])[0]
        if rows.size == 0:
            continue
        p = rank + rows[0]
        if p != rank:
            M[[rank, p]] = M[[p, rank]]
            sv[[rank, p]] = sv[[p, rank]]
        hit = np.nonzero(M[:, col])[0]
        hit = hit[hit != rank]
        M[hit] ^= M[rank]
        sv[hit] ^= sv[rank]
        pivots.append(col)
        rank += 1
    return M, sv, pivots, rank


def osd(H: np.ndarray, s: np.ndarray, post: np.ndarray, prior: np.ndarray, lam: int = 3):
    """One shot of OSD-CS of order lam: returns the correction e (n,) uint8 in qubit order and the
    index of the chosen candidate (0 = OSD-0, 1 + t = single flip of the t-th T column, after that
    the pairs)."""
    m, n = H.shape
    order = column_order(post)
    W = integer_weights(prior)[order]                         # weights in column-order coordinates
    M, sv, pivots, rank = eliminate(H, s, order)
    is_piv = np.zeros(n, dtype=bool)
    is_piv[pivots] = True
    T = np.nonzero(~is_piv)[0]
    piv = np.array(pivots, dtype=np.int64)
    s0 = sv[:rank].astype(np.int64)
    Wp = W[piv]
    cost0 = int((s0 * Wp).sum())
    d = np.where(s0 == 1, -Wp, Wp)                            # change of cost when a pivot bit flips
    best = (cost0, 0)
    cands = [()]
    for t, c in enumerate(T):
        cost = cost0 + int(W[c]) + int((M[:rank, c].astype(np.int64) * d).sum())
        cands.append((c,))
        if cost < best[0]:
            best = (cost, len(cands) - 1)
    first = T[:lam]
    for ia in range(len(first)):
        for ib in range(ia + 1, len(first)):
            a, b = first[ia], first[ib]
            flip = (M[:rank, a] ^ M[:rank, b]).astype(np.int64)
            cost = cost0 + int(W[a]) + int(W[b]) + int((flip * d).sum())
            cands.append((a, b))
            if cost < best[0]:
                best = (cost, len(cands) - 1)
    chosen = cands[best[1]]
    eS = s0.copy()
    eT = np.zeros(n, dtype=np.uint8)
    for c in chosen:
        eS ^= M[:rank, c].astype(np.int64)
        eT[c] = 1
    e_ord = eT
    e_ord[piv] = eS.astype(np.uint8)
    e = np.zeros(n, dtype=np.uint8)
    e[order] = e_ord
    return e, best[1]


def osd_batch(H, syn, post, prior, lam: int = 3, only=None):
    """osd over shots (rows of syn / post / prior); `only` selects the shots to process (the
    others get zero rows). Returns (corr (S, n) uint8, candidate index (S,), -1 where skipped)."""
    S = syn.shape[0]
    corr = np.zeros((S, H.shape[1]), dtype=np.uint8)
    idx = np.full(S, -1, dtype=np.int64)
    for i in range(S):
        if only is not None and not only[i]:
            continue
        corr[i], idx[i] = osd(H, syn[i], post[i], prior[i], lam)
    return corr, idx
