"""Seeded search for the inputs of the code construction: generating sets A, B and local code C_A.

Sec. II-A asks for symmetric sets A = A^{-1}, B = B^{-1} of size Delta that satisfy the Total
No-Conjugacy condition (ag != gb for all a, b, g, i.e. no element of B is conjugate to an
element of A); Sec. II-B asks for a classical local code C_A of length Delta, with C_B = C_A^perp
in every instance the paper builds. The paper gives no search procedure, so the one here is a
stated reading:

* a SplitMix64 stream (Steele, Lea & Flood, OOPSLA 2014) seeded with ``seed`` drives every draw;
* A is built by drawing group elements and adding either an involution or an inverse pair
  {x, x^{-1}} until |A| = Delta (identity excluded); A must generate G;
* B is built the same way from the elements whose conjugacy class meets no element of A
  (TNC) and must generate G;
* C_A is a uniformly drawn full-rank k x Delta binary generator matrix with minimum distance
  >= d_min and no all-zero coordinate (so d(C_A^perp) >= 2 and every local position is checked).

``candidate(...)`` returns the i-th accepted (A, B, C_A) of the stream. Acceptance of the
*quantum* code (k >= 1) needs the code construction, which lives with the decoder and its
oracle, so callers walk ``index = 0, 1, 2, ...`` until the built code has k >= 1.
This module holds no part of the decoder's arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .groups import Group, conjugacy_class_ids, generated_subgroup_size, group

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood 2014): state += golden gamma; output = mix(state)."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        if n <= 0:
            raise ValueError("n must be positive")
        limit = (1 << 64) - ((1 << 64) % n)
        while True:
            x = self.next()
            if x < limit:
                return x % n


def _symmetric_set(G: Group, rng: SplitMix64, delta: int, allowed: np.ndarray, max_draws: int = 100000):
    S: list[int] = []
    draws = 0
    while len(S) < delta:
        draws += 1
        if draws > max_draws:
            return None
        x = rng.below(G.order)
        if x == G.identity or not allowed[x] or x in S:
            continue
        xi = int(G.inv[x])
        if xi == x:
            S.append(x)
        elif len(S) + 2 <= delta:
            S.extend([x, xi])
    return S


def _rank_gf2(M: np.ndarray) -> int:
    M = (M.copy() & 1).astype(np.uint8)
    r = 0
    rows, cols = M.shape
    for c in range(cols):
        piv = [i for i in range(r, rows) if M[i, c]]
        if not piv:
            continue
        p = piv[0]
        M[[r, p]] = M[[p, r]]
        for i in range(rows):
            if i != r and M[i, c]:
                M[i] ^= M[r]
        r += 1
        if r == rows:
            break
    return r


def _min_distance(GA: np.ndarray) -> int:
    k, n = GA.shape
    best = n + 1
    for m in range(1, 1 << k):
        w = 0
        v = np.zeros(n, dtype=np.uint8)
        for i in range(k):
            if (m >> i) & 1:
                v ^= GA[i]
        w = int(v.sum())
        best = min(best, w)
    return best


def _local_code(rng: SplitMix64, delta: int, k: int, d_min: int, max_draws: int = 100000):
    for _ in range(max_draws):
        GA = np.array([[rng.below(2) for _ in range(delta)] for _ in range(k)], dtype=np.uint8)
        if _rank_gf2(GA) != k:
            continue
        if (GA.sum(axis=0) == 0).any():
            continue
        if _min_distance(GA) < d_min:
            continue
        return GA
    return None


@dataclass(frozen=True)
class Instance:
    """Inputs of build_code(G, A, B, C_A, C_B): group name, ordered A and B (element indices),
    the k_A x Delta generator matrix of C_A, and G_B (None means C_B = C_A^perp)."""
    group: str
    delta: int
    A: tuple
    B: tuple
    GA: np.ndarray = field(compare=False)
    GB: np.ndarray | None = field(default=None, compare=False)
    seed: int = 0
    index: int = 0

    @property
    def G(self) -> Group:
        return group(self.group)


def candidate(group_name: str, delta: int, k_A: int, d_min: int, seed: int = 0, index: int = 0,
              max_tries: int = 10000) -> Instance:
    """The ``index``-th (A, B, C_A) accepted by the seeded search described in the module doc."""
    G = group(group_name)
    cls = conjugacy_class_ids(G)
    rng = SplitMix64(seed)
    found = -1
    allowed_all = np.ones(G.order, dtype=bool)
    for _ in range(max_tries):
        A = _symmetric_set(G, rng, delta, allowed_all)
        if A is None or generated_subgroup_size(G, A) != G.order:
            continue
        a_classes = set(int(cls[a]) for a in A)
        allowed_B = np.array([int(cls[g]) not in a_classes for g in range(G.order)])
        B = _symmetric_set(G, rng, delta, allowed_B)
        if B is None or generated_subgroup_size(G, B) != G.order:
            continue
        GA = _local_code(rng, delta, k_A, d_min)
        if GA is None:
            continue
        found += 1
        if found == index:
            return Instance(group=group_name, delta=delta, A=tuple(int(a) for a in A),
                            B=tuple(int(b) for b in B), GA=GA, GB=None, seed=seed, index=index)
    raise RuntimeError(f"no candidate #{index} for {group_name} delta={delta} within {max_tries} tries")


def paper_HA() -> np.ndarray:
    """The random [6,3] parity-check matrix H_A printed in Sec. IV-B (Eq. random_matrix)."""
    return np.array([[1, 1, 0, 1, 0, 0],
                     [0, 1, 1, 0, 1, 0],
                     [1, 0, 1, 0, 0, 1]], dtype=np.uint8)


def paper_GA() -> np.ndarray:
    """Generator of C_A = ker H_A for the Sec. IV-B matrix. H_A = [M | I_3] is systematic, so
    G_A = [I_3 | M^T] spans its kernel (G_A H_A^T = M^T + M^T = 0 over GF(2))."""
    HA = paper_HA()
    M = HA[:, :3]
    return np.concatenate([np.eye(3, dtype=np.uint8), M.T.copy()], axis=1)


# Named workloads: (group, Delta, k_A, minimum distance of C_A, seed).
STANDARD = {
    "SL(2,3)": ("SL(2,3)", 4, 2, 2, 0),
    "PSL(2,7)": ("PSL(2,7)", 6, 3, 3, 0),
    "PSL(2,11)": ("PSL(2,11)", 6, 3, 3, 0),
}


def standard(name: str, index: int = 0) -> Instance:
    g, delta, k, d, seed = STANDARD[name]
    return candidate(g, delta, k, d, seed=seed, index=index)


def paper_instance(group_name: str = "PSL(2,7)", seed: int = 0, index: int = 0) -> Instance:
    """Seeded A, B on ``group_name`` with the paper's fixed C_A = ker H_A (Sec. IV-B)."""
    inst = candidate(group_name, 6, 3, 3, seed=seed, index=index)
    return Instance(group=inst.group, delta=6, A=inst.A, B=inst.B, GA=paper_GA(), GB=None,
                    seed=seed, index=index)
