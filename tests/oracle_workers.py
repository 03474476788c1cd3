"""Oracle work for the GPU parity tests, split over a process pool (started with spawn).

Only numpy and the oracle are imported here, so a worker starts quickly and never touches CUDA.
Each function recomputes its inputs from seeds and absolute shot indices, so a job is a few
integers in and the oracle's outputs back.
"""
from __future__ import annotations

import functools

import numpy as np


@functools.lru_cache(maxsize=4)
def _code(name: str):
    import workloads
    from oracle import tanner
    return tanner.from_instance(workloads.standard(name, 0))


def llr_chunk(start: int, stop: int) -> np.ndarray:
    """The oracle's lambda(p) for the binary32 bit patterns start .. stop - 1, as bit patterns."""
    from oracle import local
    u = np.arange(start, stop, dtype=np.uint32)
    return local.llr_f32(u.view(np.float32)).view(np.uint32)


def decode_shots(name: str, side: int, p: float, seed: int, shots, use_lead: bool = True, track: str = "f32"):
    """Samples the given absolute shots (X noise for side 0, Z noise for side 1) and decodes them
    with the oracle: corrections (S, n) uint8, status, iterations, posteriors (binary32) and the
    Sec. IV-A check flags. track = "f64" runs the same algorithm with FP64 priors and messages."""
    from oracle import lead as olead
    from oracle import philox
    oc = _code(name)
    shots = np.asarray(shots, dtype=np.int64)
    noise = philox.NOISE_X if side == 0 else philox.NOISE_Z
    x, z = philox.sample_errors(noise, p, seed, shots, oc.n)
    e = x if side == 0 else z
    syn = philox.syndromes(oc.sides[side].H, e)
    if track == "f64":
        corr, st, it, post = olead.decode_f64(oc, side, syn, p, use_lead=use_lead)
    else:
        corr, st, it, post = olead.decode(oc, side, syn, p, use_lead=use_lead)
    fail = olead.check(oc, side, e, corr)
    return {"corr": corr, "status": st, "iters": it, "post": post, "fail": fail}


def decode_iterated_shots(name: str, side: int, p: float, seed: int, shots, rounds: int):
    """Iterated LEAD by the oracle on the given absolute shots (X noise for side 0, Z noise for
    side 1): corrections, status, summed iterations and the Sec. IV-A check flags."""
    from oracle import lead as olead
    from oracle import philox
    oc = _code(name)
    shots = np.asarray(shots, dtype=np.int64)
    noise = philox.NOISE_X if side == 0 else philox.NOISE_Z
    x, z = philox.sample_errors(noise, p, seed, shots, oc.n)
    e = x if side == 0 else z
    syn = philox.syndromes(oc.sides[side].H, e)
    corr, st, it, _ = olead.decode_iterated(oc, side, syn, p, rounds=rounds)
    return {"corr": corr, "status": st, "iters": it, "fail": olead.check(oc, side, e, corr)}
