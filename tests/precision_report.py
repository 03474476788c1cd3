"""Per-mode precision report (GPU): error of each storage format against the FP64 oracle and the
logical error rate with its Wilson 95 % interval.

    python tests/precision_report.py [--shots 1000000] [--p 0.05] [--sample 512]

Workload: the seeded PSL(2,7) Delta=6 code, side 0, code-capacity X noise at p.
* max |dq|: the boosted local posterior table as the decoder holds it (binary32) against the
  oracle's FP64 posterior from the same weight enumerators, boosted in FP64;
* max |dlambda|: lead_local_estimate's prior LLRs, stored in each format, against the oracle's
  FP64 Phases 1-2 on `--sample` shots (absolute, and relative to |lambda|);
* LER: lead_decode in each format on `--shots` shots (the same shots for every mode), with the
  standalone min-sum baseline (binary32) beside it.
Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


from paper_2605_17796_gb300.stats import wilson95  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--shots", type=int, default=1_000_000)
    ap.add_argument("--p", type=float, default=0.05)
    ap.add_argument("--sample", type=int, default=512)
    args = ap.parse_args(argv)

    import torch
    import workloads
    from oracle import lead as olead
    from oracle import local as olocal
    from oracle import philox, tanner
    from paper_2605_17796_gb300 import lead
    from paper_2605_17796_gb300.pipeline import Pipeline

    inst = workloads.standard("PSL(2,7)", 0)
    oc = tanner.from_instance(inst)
    code = lead.Code.from_instance(inst).prepare(0)
    info = code.info
    p = args.p

    # local posterior table: binary32 on the device vs FP64 oracle
    N, N1, ml = olocal.tables(oc.sides[0].RA, oc.sides[0].RB)
    q64 = olocal.posterior_from_tables(N, N1, p)
    flip = ((ml[:, None] >> np.arange(q64.shape[1])[None, :]) & 1).astype(bool)
    q64 = np.where(flip, np.maximum(q64, 0.5), q64)
    tab = torch.zeros(q64.size, dtype=torch.float32, device="cuda")
    code.local_table(0, p, tab)
    torch.cuda.synchronize()
    dq = float(np.abs(tab.cpu().numpy().astype(np.float64).reshape(q64.shape) - q64).max())

    # prior LLRs per mode on a sample of shots
    x, _ = philox.sample_errors(philox.NOISE_X, p, 9, np.arange(args.sample), oc.n)
    syn = philox.syndromes(oc.HZ, x)
    _, lam64 = olead.prior_f64(oc, 0, syn, p)
    sd = torch.from_numpy(philox.pack_bits(syn, info.words_m[0]).view(np.int32)).cuda()
    modes = {"fp32": 0, "bf16": 1, "fp16": 2}
    report = {"workload": f"PSL(2,7) Delta=6 side 0, X noise p={p}", "max_abs_dq": dq, "modes": {}}
    pipe = Pipeline(code, 1 << 20, 0)
    for name, prec in modes.items():
        o = lead.opts(side=0, p=p, precision=prec)
        ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
        out = torch.zeros((args.sample, info.n), dtype=torch.float32 if prec == 0 else torch.int16, device="cuda")
        code.local_estimate(o, sd, args.sample, out, ws)
        torch.cuda.synchronize()
        raw = out.cpu().numpy()
        if prec == 0:
            lam = raw.astype(np.float64)
        elif prec == 1:
            lam = (raw.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        else:
            lam = raw.view(np.float16).astype(np.float64)
        d = np.abs(lam - lam64)
        r = pipe.run(lead.NOISE_X, p, args.shots, seed=5, offset=0, precision=prec)
        report["modes"][name] = {"max_abs_dlambda": float(d.max()),
                                 "max_rel_dlambda": float((d / np.maximum(np.abs(lam64), 1e-30)).max()),
                                 "ler": r.failures / args.shots, "ler_ci95": wilson95(r.failures, args.shots),
                                 "mean_iters": r.iters_sum / args.shots, "shots": args.shots}
    r = pipe.run(lead.NOISE_X, p, args.shots, seed=5, offset=0, use_lead=False)
    report["min_sum_baseline_fp32"] = {"ler": r.failures / args.shots, "ler_ci95": wilson95(r.failures, args.shots),
                                       "mean_iters": r.iters_sum / args.shots}
    print(json.dumps(report))


if __name__ == "__main__":
    main()
