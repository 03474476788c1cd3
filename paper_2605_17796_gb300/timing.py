"""Time the library's kernels on one synthetic batch (CUDA events on the current stream).

    python -m paper_2605_17796_gb300.timing --code PSL(2,7) --shots 65536 --p 0.05 --reps 3

Samples X noise, then times lead_decode (LEAD or, with --baseline, plain min-sum) and
lead_local_estimate on the same syndromes, in the storage format of --precision (0 binary32,
1 bfloat16, 2 binary16); with --priors also the per-qubit-prior path (priors drawn uniformly
from [p/2, 3p/2]); with --osd K also OSD-CS of order K on the shots min-sum leaves unconverged. Used for kernel tuning and for small ncu captures.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--code", default="PSL(2,7)")
    ap.add_argument("--shots", type=int, default=65536)
    ap.add_argument("--p", type=float, default=0.05)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--baseline", action="store_true")
    ap.add_argument("--skip-local", action="store_true")
    ap.add_argument("--skip-decode", action="store_true")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--priors", action="store_true")
    ap.add_argument("--osd", type=int, default=None, help="also time OSD-CS of this order after decode")
    ap.add_argument("--autotune", type=int, default=0, help="autotune the decode kernel on this many shots first")
    ap.add_argument("--report", action="store_true", help="print the min-sum kernels' compile report")
    args = ap.parse_args(argv)

    import torch
    import workloads
    from . import lead

    inst = workloads.standard(args.code, 0)
    code = lead.Code.from_instance(inst)
    if args.report:
        print(code.compile())
    code.prepare(0)
    if args.autotune:
        print(code.autotune(0, args.precision, args.p, args.autotune))
    info = code.info
    shots = args.shots
    ex = torch.zeros((shots, info.words_n), dtype=torch.int32, device="cuda")
    sz = torch.zeros((shots, info.words_m[0]), dtype=torch.int32, device="cuda")
    code.sample(lead.NOISE_X, args.p, shots, 0, 0, err_x=ex, syn_z=sz)
    o = lead.opts(side=0, p=args.p, use_lead=not args.baseline, precision=args.precision)
    ws = torch.zeros(max(code.workspace_bytes(lead.opts(side=0, p=args.p)), 256) // 4 + 64,
                     dtype=torch.int32, device="cuda")
    corr = torch.zeros_like(ex)
    st = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    it = torch.zeros(shots, dtype=torch.int32, device="cuda")

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for _ in range(0 if args.skip_decode else args.reps):
        ms = timed(lambda: code.decode(o, sz, shots, corr, st, it, workspace=ws))
        si = int(it.sum())
        print(f"decode {args.code} {shots} shots p={args.p} {'baseline' if args.baseline else 'LEAD'}: "
              f"{ms:.3f} ms, {shots / ms * 1e3:.3e} shots/s, {si} shot-iterations, "
              f"{si / ms * 1e3:.3e} shot-iterations/s")
    if not args.skip_local:
        esize = 4 if args.precision == lead.PREC_FP32 else 2
        llr = torch.zeros((shots, info.n), dtype=torch.float32 if esize == 4 else torch.int16, device="cuda")
        lo = lead.opts(side=0, p=args.p, precision=args.precision)
        for _ in range(args.reps):
            ms = timed(lambda: code.local_estimate(lo, sz, shots, llr, ws))
            nbytes = shots * (info.n * esize + info.words_m[0] * 4)
            print(f"local_estimate {args.code} {shots} shots precision {args.precision}: {ms:.3f} ms, "
                  f"{shots / ms * 1e3:.3e} shots/s, {nbytes / ms / 1e6:.1f} GB/s algorithmic")
    if args.osd is not None:
        post = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
        prior = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
        ows = torch.zeros(code.osd_workspace_bytes(o, shots) // 4 + 64, dtype=torch.int32, device="cuda")
        for _ in range(args.reps):
            code.decode(o, sz, shots, corr, st, it, llr=post, workspace=ws)
            if not args.baseline:
                code.local_estimate(lead.opts(side=0, p=args.p), sz, shots, prior, ws)
            torch.cuda.synchronize()
            todo = int(((st & lead.ST_CONVERGED) == 0).sum())
            ms = timed(lambda: code.osd(o, args.osd, sz, shots, post, st, corr,
                                        prior=None if args.baseline else prior, workspace=ows))
            print(f"osd {args.code} order {args.osd}: {todo} of {shots} shots unconverged, {ms:.3f} ms, "
                  f"{todo / ms * 1e3:.3e} post-processed shots/s")
    if args.priors:
        prior = torch.rand((shots, info.n), generator=torch.Generator(device="cuda").manual_seed(1),
                           device="cuda") * args.p + 0.5 * args.p
        lam = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
        pws = torch.zeros(code.priors_workspace_bytes(o, shots) // 4 + 64, dtype=torch.int32, device="cuda")
        for _ in range(args.reps):
            ms = timed(lambda: code.local_estimate_priors(o, sz, shots, prior, lam, workspace=pws))
            print(f"local_estimate_priors {args.code} {shots} shots: {ms:.3f} ms, {shots / ms * 1e3:.3e} shots/s, "
                  f"{shots * info.order / ms * 1e3:.3e} vertex-items/s")


if __name__ == "__main__":
    main()
