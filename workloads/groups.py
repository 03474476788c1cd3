"""Finite groups used as the vertex sets of the left-right Cayley complex (Sec. II-A).

The decoder's code instances are built on SL(2, F_q) and PSL(2, F_q) for small primes q.
This module only *enumerates* those groups and writes their Cayley tables; it holds none of
LEAD's arithmetic. A group is returned as a ``Group`` with

* ``mul[i, j]``  index of the product  g_i * g_j  (row-major |G| x |G| int32 table),
* ``inv[i]``     index of g_i^{-1},
* ``identity``   index of the identity,
* ``elems``      the 2x2 matrices (canonical representatives for PSL) as a (|G|, 4) array.

Element order is the lexicographic order of the canonical matrix tuple (a, b, c, d), which
makes every table a deterministic function of (kind, q).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Group:
    name: str
    mul: np.ndarray       # (|G|, |G|) int32
    inv: np.ndarray       # (|G|,) int32
    identity: int
    elems: np.ndarray     # (|G|, 4) int64, matrix entries (a, b, c, d) of [[a, b], [c, d]]

    @property
    def order(self) -> int:
        return int(self.mul.shape[0])


def _canonical_psl(t, q):
    """Canonical representative of the coset {M, -M}: the lexicographically smaller tuple."""
    neg = tuple((-x) % q for x in t)
    return min(t, neg)


def special_linear(q: int, projective: bool) -> Group:
    """SL(2, F_q) (projective=False) or PSL(2, F_q) = SL(2, F_q)/{+-I} (projective=True), q prime."""
    if q < 2 or any(q % d == 0 for d in range(2, int(q ** 0.5) + 1)):
        raise ValueError("q must be prime")
    mats = []
    for a in range(q):
        for b in range(q):
            for c in range(q):
                for d in range(q):
                    if (a * d - b * c) % q == 1:
                        t = (a, b, c, d)
                        if projective:
                            t = _canonical_psl(t, q)
                        mats.append(t)
    mats = sorted(set(mats))
    index = {t: i for i, t in enumerate(mats)}
    n = len(mats)
    E = np.array(mats, dtype=np.int64)
    a, b, c, d = E[:, 0], E[:, 1], E[:, 2], E[:, 3]
    # product [[a1,b1],[c1,d1]] @ [[a2,b2],[c2,d2]]
    pa = (a[:, None] * a[None, :] + b[:, None] * c[None, :]) % q
    pb = (a[:, None] * b[None, :] + b[:, None] * d[None, :]) % q
    pc = (c[:, None] * a[None, :] + d[:, None] * c[None, :]) % q
    pd = (c[:, None] * b[None, :] + d[:, None] * d[None, :]) % q
    mul = np.empty((n, n), dtype=np.int32)
    for i in range(n):
        for j in range(n):
            t = (int(pa[i, j]), int(pb[i, j]), int(pc[i, j]), int(pd[i, j]))
            if projective:
                t = _canonical_psl(t, q)
            mul[i, j] = index[t]
    ident = (1, 0, 0, 1)
    if projective:
        ident = _canonical_psl(ident, q)
    e = index[ident]
    inv = np.empty(n, dtype=np.int32)
    for i in range(n):
        inv[i] = int(np.nonzero(mul[i] == e)[0][0])
    name = ("PSL" if projective else "SL") + f"(2,{q})"
    return Group(name=name, mul=mul, inv=inv, identity=e, elems=E)


_CACHE: dict = {}


def group(name: str) -> Group:
    """Group by name: 'SL(2,3)', 'PSL(2,7)', 'PSL(2,11)', ... (cached)."""
    if name not in _CACHE:
        key = name.replace(" ", "")
        if key.startswith("SL(2,") and key.endswith(")"):
            _CACHE[name] = special_linear(int(key[5:-1]), projective=False)
        elif key.startswith("PSL(2,") and key.endswith(")"):
            _CACHE[name] = special_linear(int(key[6:-1]), projective=True)
        else:
            raise ValueError(f"unknown group {name!r}")
    return _CACHE[name]


def conjugacy_class_ids(G: Group) -> np.ndarray:
    """cls[i] = id of the conjugacy class of g_i (ids in order of first appearance)."""
    n = G.order
    cls = -np.ones(n, dtype=np.int64)
    nxt = 0
    for i in range(n):
        if cls[i] >= 0:
            continue
        # orbit of g_i under conjugation h g h^{-1}
        orbit = G.mul[G.mul[np.arange(n), i], G.inv]  # h * g_i * h^{-1} for all h
        cls[orbit] = nxt
        nxt += 1
    return cls


def generated_subgroup_size(G: Group, gens) -> int:
    """|<gens>| by closure under right multiplication."""
    seen = np.zeros(G.order, dtype=bool)
    seen[G.identity] = True
    frontier = [G.identity]
    gens = list(gens)
    while frontier:
        nf = []
        for x in frontier:
            for s in gens:
                y = int(G.mul[x, s])
                if not seen[y]:
                    seen[y] = True
                    nf.append(y)
        frontier = nf
    return int(seen.sum())
