"""Philox4x32-10 counter-based generator and the noise models of Sec. IV-A (oracle only).

Philox4x32-10 as published by Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
as 1, 2, 3" (SC'11): a 4-word counter and a 2-word key; each of the 10 rounds multiplies
counter words 0 and 2 by the constants M0 = 0xD2511F53 and M1 = 0xCD9E8D57, and permutes and
XORs the high/low product halves with the other words and the round key; the key is bumped by
the Weyl constants W0 = 0x9E3779B9, W1 = 0xBB67AE85 between rounds.

Draw layout (a reading: the paper does not say how errors are sampled). The 32-bit uniform
for qubit i of shot s is word (i mod 4) of Philox(counter = (i div 4, s mod 2^32, s div 2^32,
0), key = (seed mod 2^32, seed div 2^32)); shot indices are absolute (shot_offset + local).

Noise (Sec. IV-A uses depolarizing noise; the workloads also use code-capacity X noise):
* Bernoulli(p):  the qubit flips iff u < floor(p * 2^32).
* depolarizing(p): with t1 = floor((p/3) 2^32), t2 = floor((2p/3) 2^32), t3 = floor(p 2^32),
  u < t1 is X, t1 <= u < t2 is Y, t2 <= u < t3 is Z, otherwise I. The X part is X or Y
  (u < t2), the Z part is Y or Z (t1 <= u < t3).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 on uint64 arrays holding 32-bit values. Returns 4 arrays."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3))
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c0                     # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
    return c0, c1, c2, c3


def uniforms(seed: int, shots, n: int) -> np.ndarray:
    """u[s, i] (uint64 holding a 32-bit value) for absolute shot indices ``shots`` and qubits 0..n-1."""
    shots = np.asarray(shots, dtype=np.uint64).reshape(-1, 1)
    groups = np.arange((n + 3) // 4, dtype=np.uint64).reshape(1, -1)
    c0 = np.broadcast_to(groups, (shots.shape[0], groups.shape[1]))
    c1 = np.broadcast_to(shots & _MASK32, c0.shape)
    c2 = np.broadcast_to(shots >> np.uint64(32), c0.shape)
    c3 = np.zeros_like(c0)
    words = philox4x32_10(c0, c1, c2, c3, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u = np.stack(words, axis=-1).reshape(shots.shape[0], -1)
    return u[:, :n]


def thresholds(p: float):
    """Integer thresholds of the two noise models (computed in IEEE double, then floored)."""
    if not (0.0 <= p < 1.0):
        raise ValueError("p must be in [0, 1)")
    two32 = 4294967296.0
    t_bern = int(np.floor(p * two32))
    t1 = int(np.floor((p / 3.0) * two32))
    t2 = int(np.floor(((2.0 * p) / 3.0) * two32))
    t3 = t_bern
    return t_bern, (t1, t2, t3)


NOISE_X, NOISE_Z, NOISE_DEPOL = 0, 1, 2


def sample_errors(noise: int, p: float, seed: int, shots, n: int):
    """Error bits (0/1 uint8) for absolute shot indices: returns (x_part, z_part), each (S, n)."""
    u = uniforms(seed, shots, n)
    tb, (t1, t2, t3) = thresholds(p)
    zero = np.zeros(u.shape, dtype=np.uint8)
    if noise == NOISE_X:
        return (u < np.uint64(tb)).astype(np.uint8), zero
    if noise == NOISE_Z:
        return zero, (u < np.uint64(tb)).astype(np.uint8)
    if noise == NOISE_DEPOL:
        xp = (u < np.uint64(t2)).astype(np.uint8)
        zp = ((u >= np.uint64(t1)) & (u < np.uint64(t3))).astype(np.uint8)
        return xp, zp
    raise ValueError("unknown noise model")


def syndromes(H: np.ndarray, e: np.ndarray) -> np.ndarray:
    """s = H e mod 2 for each row of e (S, n) -> (S, m) uint8."""
    return ((e.astype(np.int64) @ H.T.astype(np.int64)) & 1).astype(np.uint8)


def pack_bits(b: np.ndarray, words: int) -> np.ndarray:
    """(S, nbits) 0/1 -> (S, words) uint32 with bit j of word w = entry 32 w + j."""
    S, nb = b.shape
    out = np.zeros((S, words), dtype=np.uint32)
    for j in range(nb):
        out[:, j >> 5] |= (b[:, j].astype(np.uint32) << np.uint32(j & 31))
    return out


def unpack_bits(w: np.ndarray, nbits: int) -> np.ndarray:
    w = np.asarray(w, dtype=np.uint32)
    j = np.arange(nbits)
    return ((w[:, j >> 5] >> (j & 31).astype(np.uint32)) & 1).astype(np.uint8)
