"""Serving workload on the continuous-batching decode server (lead_server_*).

Requests are single shots under depolarizing noise (both sides decoded, each with the marginal
prior 2p/3), drawn from several codes with a given mix, arriving as a Poisson process. The
syndromes are produced on the device by lead_sample and copied to the host beforehand; the
server admits each request at its arrival time. Latency = completion seen by the dispatcher -
arrival, on the server's clock.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import lead


def request_rows(code: lead.Code, p: float, n: int, seed: int, offset: int = 0) -> np.ndarray:
    """(n, words_m[0] + words_m[1]) uint32 host rows of depolarizing syndromes (side 0, side 1)."""
    info = code.info
    dev = torch.device("cuda", info.prepared_device)
    sz = torch.zeros((n, info.words_m[0]), dtype=torch.int32, device=dev)
    sx = torch.zeros((n, info.words_m[1]), dtype=torch.int32, device=dev)
    code.sample(lead.NOISE_DEPOL, p, n, seed, offset, syn_z=sz, syn_x=sx)
    return torch.cat([sz, sx], dim=1).cpu().numpy().view(np.uint32)


def poisson_trace(rate: float, n: int, mix, rng: np.random.Generator):
    """Arrival offsets (ns) of a Poisson process with `rate` requests/s and the code of each."""
    gaps = rng.exponential(1.0 / rate, n)
    t = np.cumsum(gaps) * 1e9
    codes = rng.choice(len(mix), size=n, p=np.asarray(mix) / np.sum(mix))
    return t.astype(np.int64), codes.astype(np.int32)


def run_trace(server: lead.Server, rows_per_code, arrival_ns, code_of, lead_ns: int = 200_000_000,
              timeout_s: float = 120.0):
    """Submits every request ahead of time (arrival = start + lead_ns + its offset; lead_ns
    leaves time for the submission itself) and collects all results.
    Returns (results, corrections) ordered by request id."""
    n = len(arrival_ns)
    t0 = server.clock_ns() + lead_ns
    nxt = np.zeros(len(rows_per_code), dtype=np.int64)
    idx_in_code = np.zeros(n, dtype=np.int64)
    for c in range(len(rows_per_code)):
        sel = np.nonzero(code_of == c)[0]
        idx_in_code[sel] = np.arange(sel.size)
        if sel.size:
            server.submit(c, rows_per_code[c][idx_in_code[sel]], sel.astype(np.uint64), t0 + arrival_ns[sel])
        nxt[c] = sel.size
    results = []
    corrs = []
    deadline = time.time() + timeout_s
    got = 0
    while got < n:
        r, cr = server.poll()
        if len(r):
            results.append(r)
            corrs.append(cr)
            got += len(r)
        else:
            if time.time() > deadline:
                raise TimeoutError(f"server returned {got} of {n} results")
            time.sleep(0.0005)
    res = np.concatenate(results)
    cor = np.concatenate(corrs)
    order = np.argsort(res["id"])
    return res[order], cor[order]


def latency_stats(res, rate: float):
    lat = (res["done_ns"] - res["arrival_ns"]) / 1e3
    span = (res["done_ns"].max() - res["arrival_ns"].min()) / 1e9
    return {"requests": int(len(res)), "offered_rate": rate, "throughput": float(len(res) / span),
            "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
            "max_us": float(lat.max()), "mean_us": float(lat.mean())}
