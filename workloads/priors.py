"""Seeded per-qubit prior probabilities and errors drawn from them (inputs only).

A prior p_i is drawn per shot and qubit uniformly from [(1 - spread) p, (1 + spread) p] (a
channel whose strength varies across qubits and shots around the marginal p); the error bit of
the qubit is then Bernoulli(p_i). Both come from numpy's PCG64 with the given seed.
"""
from __future__ import annotations

import numpy as np


def per_qubit_priors(shots: int, n: int, p: float, spread: float = 0.5, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    lo, hi = (1.0 - spread) * p, (1.0 + spread) * p
    return rng.uniform(lo, hi, size=(shots, n)).astype(np.float32)


def errors_from_priors(prior: np.ndarray, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed ^ 0x5EED)
    return (rng.random(prior.shape) < prior.astype(np.float64)).astype(np.uint8)
