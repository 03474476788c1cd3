"""Left-right Cayley complex and quantum Tanner code (Sec. II-A, II-B); oracle only.

Readings of the paper fixed here (each also listed in the design notes):

* Faces (Eq. group_set): the face of (g, a, b) is {(g,0), (ag,1), (gb,1), (agb,0)}. The same
  face arises from (agb, a^{-1}, b^{-1}); the qubit is the canonical (smaller) of the two
  tuples (g, index(a), index(b)), and qubits are numbered in sorted canonical order.
* Local views phi_v: Q(v) -> A x B. A V0 vertex g sees face (g, a, b) at local position
  (a, b). A V1 vertex h sees at (a, b) the face {(h,1), (ah,0), (hb,0), (ahb,1)}, which is the
  V0-form face (ah, a^{-1}, b). Local index j = index(b) * Delta + index(a) (column-major; the
  worked example of Appendix A, Eq. product, equals kron(H_B, H_A) in this order).
* Local checks: Z-generators on V0 are a basis of C_A (x) C_B, i.e. the rows of
  kron(G_B, G_A); X-generators on V1 are a basis of C_A^perp (x) C_B^perp, the rows of
  kron(H_B, H_A). G_A is the generator given by the caller, G_B the caller's generator of C_B
  or, if none is given, the canonical (RREF) basis of C_A^perp (C_B = C_A^perp, the choice of
  every instance in Sec. IV); H_A and H_B are the RREF bases of C_A^perp and C_B^perp.
* Global check index of local row r at vertex v is v * m_l + r.
* Side 0 decodes X errors with H_Z (V0 views), side 1 decodes Z errors with H_X (V1 views).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import gf2


@dataclass
class Side:
    """One decoding side: checks H (m x n, 0/1), local check matrix L (m_l x Delta^2),
    views[v, j] -> qubit, and for every qubit its two (vertex, local index) views."""
    H: np.ndarray
    L: np.ndarray
    RA: np.ndarray          # row factor of L = kron(RB, RA) acting on the A coordinate
    RB: np.ndarray          # row factor acting on the B coordinate
    views: np.ndarray       # (|G|, Delta^2) int64
    qubit_views: np.ndarray  # (n, 2, 2): [i, t] = (vertex, local index), t=0 the smaller vertex

    @property
    def m_l(self) -> int:
        return int(self.L.shape[0])


@dataclass
class TannerCode:
    order: int
    delta: int
    n: int
    faces: np.ndarray       # (n, 3) canonical (g, ia, ib)
    sides: tuple            # (Side for X errors / H_Z, Side for Z errors / H_X)
    k: int
    rank_HZ: int
    rank_HX: int

    @property
    def HZ(self):
        return self.sides[0].H

    @property
    def HX(self):
        return self.sides[1].H


def check_generating_sets(mul, inv, identity, A, B):
    """Sec. II-A: A = A^{-1}, B = B^{-1}, identity excluded, and TNC (ag != gb for all a,b,g)."""
    A = list(A)
    B = list(B)
    if len(set(A)) != len(A) or len(set(B)) != len(B):
        raise ValueError("A and B must not repeat elements")
    if identity in A or identity in B:
        raise ValueError("identity in a generating set")
    if set(int(inv[a]) for a in A) != set(A) or set(int(inv[b]) for b in B) != set(B):
        raise ValueError("A or B is not closed under inversion")
    order = mul.shape[0]
    for g in range(order):
        for a in A:
            ag = mul[a, g]
            for b in B:
                if ag == mul[g, b]:
                    raise ValueError("TNC violated: ag == gb")


def build(mul, inv, identity, A, B, GA, GB=None) -> TannerCode:
    """The quantum Tanner code of Sec. II from a Cayley table and the local codes."""
    mul = np.asarray(mul, dtype=np.int64)
    inv = np.asarray(inv, dtype=np.int64)
    A = [int(a) for a in A]
    B = [int(b) for b in B]
    delta = len(A)
    if len(B) != delta:
        raise ValueError("|A| must equal |B|")
    check_generating_sets(mul, inv, identity, A, B)
    order = mul.shape[0]
    GA = np.asarray(GA, dtype=np.uint8) & 1
    if GA.shape[1] != delta or gf2.rank(GA) != GA.shape[0]:
        raise ValueError("G_A must be full rank with Delta columns")
    if GB is None:
        GB = gf2.dual_basis(GA)
    GB = np.asarray(GB, dtype=np.uint8) & 1
    if GB.shape[1] != delta or gf2.rank(GB) != GB.shape[0]:
        raise ValueError("G_B must be full rank with Delta columns")
    HA = gf2.dual_basis(GA)
    HB = gf2.dual_basis(GB)

    a_idx = {a: i for i, a in enumerate(A)}
    b_idx = {b: i for i, b in enumerate(B)}
    a_inv = [a_idx[int(inv[a])] for a in A]
    b_inv = [b_idx[int(inv[b])] for b in B]

    # canonical faces
    canon = {}
    for g in range(order):
        for ia, a in enumerate(A):
            for ib, b in enumerate(B):
                other = (int(mul[mul[a, g], b]), a_inv[ia], b_inv[ib])
                canon[(g, ia, ib)] = min((g, ia, ib), other)
    faces = sorted(set(canon.values()))
    qid = {f: i for i, f in enumerate(faces)}
    n = len(faces)

    views0 = np.empty((order, delta * delta), dtype=np.int64)
    views1 = np.empty((order, delta * delta), dtype=np.int64)
    for v in range(order):
        for ia in range(delta):
            for ib in range(delta):
                j = ib * delta + ia
                views0[v, j] = qid[canon[(v, ia, ib)]]
                g1 = int(mul[A[ia], v])          # V1 vertex v sees the V0-form face (a v, a^-1, b)
                views1[v, j] = qid[canon[(g1, a_inv[ia], ib)]]

    sides = []
    for views, RA, RB in ((views0, GA, GB), (views1, HA, HB)):
        L = np.kron(RB, RA).astype(np.uint8)
        m_l = L.shape[0]
        H = np.zeros((order * m_l, n), dtype=np.uint8)
        for v in range(order):
            for r in range(m_l):
                cols = views[v, L[r] == 1]
                H[v * m_l + r, cols] ^= 1
        qv = [[] for _ in range(n)]
        for v in range(order):
            for j in range(delta * delta):
                qv[views[v, j]].append((v, j))
        if any(len(x) != 2 for x in qv):
            raise ValueError("a qubit does not lie in exactly two views of one side")
        qubit_views = np.array([sorted(x) for x in qv], dtype=np.int64)
        sides.append(Side(H=H, L=L, RA=RA, RB=RB, views=views, qubit_views=qubit_views))

    rZ = gf2.rank(sides[0].H)
    rX = gf2.rank(sides[1].H)
    return TannerCode(order=order, delta=delta, n=n, faces=np.array(faces, dtype=np.int64),
                      sides=tuple(sides), k=n - rZ - rX, rank_HZ=rZ, rank_HX=rX)


def from_instance(inst) -> TannerCode:
    G = inst.G
    return build(G.mul, G.inv, G.identity, inst.A, inst.B, inst.GA, inst.GB)
