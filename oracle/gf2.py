"""Plain GF(2) linear algebra on 0/1 uint8 matrices (oracle; test infrastructure only)."""
from __future__ import annotations

import numpy as np


def rref(M: np.ndarray):
    """Reduced row echelon form over GF(2). Returns (R, pivots) with R's zero rows removed.

    The RREF of a matrix depends only on its row space, so it is the canonical basis used
    wherever a basis of a code or of its dual must be chosen. Rows are bit-packed only to
    make the row XORs cheap; the elimination is the textbook Gauss-Jordan sweep."""
    M = np.asarray(M, dtype=np.uint8) & 1
    rows, cols = M.shape
    P = np.packbits(M, axis=1)                   # bit c of a row -> byte c>>3, bit 7-(c&7)
    pivots = []
    r = 0
    for c in range(cols):
        if r == rows:
            break
        byte, mask = c >> 3, np.uint8(0x80 >> (c & 7))
        col = (P[:, byte] & mask) != 0
        nz = np.nonzero(col[r:])[0]
        if nz.size == 0:
            continue
        p = r + int(nz[0])
        if p != r:
            P[[r, p]] = P[[p, r]]
            col[[r, p]] = col[[p, r]]
        hit = np.nonzero(col)[0]
        hit = hit[hit != r]
        if hit.size:
            P[hit] ^= P[r]
        pivots.append(c)
        r += 1
    R = np.unpackbits(P[:r], axis=1, count=cols).astype(np.uint8)
    return R, pivots


def rank(M: np.ndarray) -> int:
    return len(rref(M)[1])


def kernel_basis(M: np.ndarray) -> np.ndarray:
    """A basis of {x : M x = 0} as rows, in RREF (canonical)."""
    M = np.asarray(M, dtype=np.uint8)
    cols = M.shape[1]
    R, piv = rref(M)
    free = [c for c in range(cols) if c not in set(piv)]
    basis = []
    for f in free:
        x = np.zeros(cols, dtype=np.uint8)
        x[f] = 1
        for i, pc in enumerate(piv):
            x[pc] = R[i, f]
        basis.append(x)
    if not basis:
        return np.zeros((0, cols), dtype=np.uint8)
    return rref(np.array(basis, dtype=np.uint8))[0]


def dual_basis(G: np.ndarray) -> np.ndarray:
    """Canonical (RREF) basis of the dual code of the row space of G."""
    return kernel_basis(G)


class RowSpace:
    """Membership test for the row space of a matrix (reduce by its RREF)."""

    def __init__(self, M: np.ndarray):
        self.R, self.piv = rref(M)

    def contains(self, x: np.ndarray) -> bool:
        x = (np.asarray(x, dtype=np.uint8) & 1).copy()
        for i, c in enumerate(self.piv):
            if x[c]:
                x ^= self.R[i]
        return not x.any()
