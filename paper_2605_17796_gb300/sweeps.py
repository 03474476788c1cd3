"""Logical-error-rate sweeps over the scaling parameter alpha (Phase 2, Sec. III-B and IV-C).

    python -m paper_2605_17796_gb300.sweeps --code "PSL(2,7)" --p 0.005,0.01,0.02,0.03 \
        --alpha 1,0.5,0.1,0.01 --shots 200000 [--noise x|depol] [--precision 0]

For every (alpha, p) it decodes the same seeded shots with LEAD and prints one JSON line: the
logical error rate with its Wilson 95 % interval, the fraction of shots whose min-sum did not
converge, the mean global iterations, and the code's parameters (n, k, Delta, A, B, the
generator of C_A and the seeded search that chose them). One line per p is added for the standalone min-sum
baseline (alpha = null) on the same shots. Sec. IV-C's experiment is alpha = 1 against
alpha = 0.01 across the noise range. --estimator minsum uses local min-sum BP as the Phase-1
local decoder instead of the exact posterior; --osd ORDER adds OSD-CS of that order after
min-sum (the paper's BP-OSD global decoder), for LEAD and the baseline alike. --rounds R > 1
runs iterated LEAD (an extension): up to R - 1 further rounds on the unconverged shots, each
with the last global posterior as per-qubit prior; for the baseline the same rounds restart
min-sum from that prior without the local stage.

The normalised iteration count of Sec. IV-A, I = I_g + I_l m_l / m_g, is reported with I_l
summed over the |G| parallel local decoders of a shot (m_g = |G| m_l), i.e. I_l m_l / m_g is
the expected local iterations per vertex: sum_s P(s) I_l(s) over local syndromes s, with
P(s) from the coset weight enumerators (exact, not sampled). X noise only (one side).
"""
from __future__ import annotations

import argparse
import json

from . import lead
from .pipeline import Pipeline
from .stats import wilson95  # noqa: F401  (re-exported for callers of this module)




def expected_local_iterations(code: lead.Code, side: int, p: float, estimator: int) -> float:
    """sum_s P(s) I_l(s) for one side under i.i.d. flips with probability p (see the module doc)."""
    import numpy as np
    import torch
    info = code.info
    S, nl = 1 << info.m_l[side], info.delta ** 2
    dev = torch.device("cuda", info.prepared_device)
    t = torch.empty(S * nl, dtype=torch.float32, device=dev)
    it = torch.empty(S, dtype=torch.int32, device=dev)
    code.local_table_est(side, p, estimator, t, it)
    iters = (it.cpu().numpy() & 0xFFFF).astype(np.float64)
    N, _, _ = code.enumerators(side)
    w = np.arange(nl + 1)
    ps = (N.astype(np.float64) * (p ** w) * ((1.0 - p) ** (nl - w))).sum(axis=1)
    return float((ps * iters).sum())


def sweep(code: lead.Code, ps, alphas, shots: int, noise: int = lead.NOISE_X, precision: int = lead.PREC_FP32,
          chunk: int = 1 << 18, seed: int = 0, baseline: bool = True, estimator: int = lead.EST_EXACT,
          osd_order=None, rounds: int = 1):
    """Yields one result dict per (alpha, p) and, with baseline, per p for plain min-sum."""
    pipe = Pipeline(code, min(chunk, shots), code.info.prepared_device)
    configs = [(a, True) for a in alphas] + ([(None, False)] if baseline else [])
    for p in ps:
        il = expected_local_iterations(code, 0, p, estimator) if noise == lead.NOISE_X else None
        for alpha, use_lead in configs:
            r = pipe.run(noise, p, shots, seed=seed, offset=0, alpha=alpha if alpha else 1.0, use_lead=use_lead,
                         precision=precision, estimator=estimator, osd_order=osd_order, rounds=rounds)
            ig = r.iters_sum / shots
            row = {"p": p, "alpha": alpha, "decoder": "LEAD" if use_lead else "min-sum", "shots": shots,
                   "ler": r.failures / shots, "ler_ci95": wilson95(r.failures, shots),
                   "not_converged": r.not_converged / shots, "mean_iters": ig, "precision": precision,
                   "estimator": ("minsum" if estimator == lead.EST_MINSUM else "exact") if use_lead else None,
                   "osd_order": osd_order, "rounds": rounds}
            if use_lead and il is not None:
                row["local_iters_per_vertex"] = il
                row["normalized_iters"] = ig + il
            yield row


def main(argv=None):
    import workloads

    ap = argparse.ArgumentParser()
    ap.add_argument("--code", default="PSL(2,7)")
    ap.add_argument("--p", default="0.005,0.01,0.015,0.02,0.03")
    ap.add_argument("--alpha", default="1,0.5,0.1,0.01")
    ap.add_argument("--shots", type=int, default=200_000)
    ap.add_argument("--noise", choices=["x", "depol"], default="x")
    ap.add_argument("--precision", type=int, default=lead.PREC_FP32)
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--estimator", choices=["exact", "minsum"], default="exact")
    ap.add_argument("--osd", type=int, default=None)
    ap.add_argument("--rounds", type=int, default=1)
    ap.add_argument("--chunk", type=int, default=1 << 16)
    args = ap.parse_args(argv)
    inst = workloads.standard(args.code, 0)
    code = lead.Code.from_instance(inst).prepare(0)
    params = {"n": code.info.n, "k": code.info.k, "delta": inst.delta, "A": list(inst.A), "B": list(inst.B),
              "C_A": inst.GA.astype(int).tolist(), "search_seed": inst.seed, "search_index": inst.index}
    noise = lead.NOISE_X if args.noise == "x" else lead.NOISE_DEPOL
    ps = [float(x) for x in args.p.split(",")]
    alphas = [float(x) for x in args.alpha.split(",")]
    est = lead.EST_MINSUM if args.estimator == "minsum" else lead.EST_EXACT
    for row in sweep(code, ps, alphas, args.shots, noise, args.precision, chunk=args.chunk,
                     baseline=not args.no_baseline, estimator=est, osd_order=args.osd, rounds=args.rounds):
        row["code"] = args.code
        row["code_params"] = params
        row["noise"] = args.noise
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
