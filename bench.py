"""Benchmark of the LEAD decoding path on GB300 (one JSON line on rank 0).

Workload: the seeded PSL(2,7) quantum Tanner code (|G| = 168, Delta = 6, C_A a seeded [6,3,3]
code, C_B = C_A^perp, n = 3024), code-capacity X noise at p = 0.01, 0.02, ..., 0.10 with
``--shots-per-p`` shots each (10^6 by default), LEAD with alpha = 1 and at most 32 global
min-sum iterations. One step = the whole sweep: sample, decode (local estimation, merge,
min-sum with a per-iteration syndrome check), residual/logical check. Every chunk of 2^20 shots
holds more than the 129 MB L2 (errors alone are 400 MB), so no L2 flush is needed.

``--impl reference`` times the CPU oracle (the only reference that exists: the paper ships no
code) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P_SWEEP = [round(0.01 * i, 2) for i in range(1, 11)]
WORKLOAD = "PSL(2,7)"
PSL11_P = 0.0267          # X marginal 2p/3 of depolarizing p = 0.04, as in the multi-code batch
TUNE_P = (0.01, 0.02, 0.03, 0.04, 0.05)   # priors the min-sum kernel's launch shape is tuned at
METRIC = "shots decoded/s at matched logical error rate; p50/p99 decode latency (µs)"
UNIT = "shots/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _clock_sampler(path):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        return subprocess.Popen(cmd, stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except OSError:
        return None


def _clock_summary(path, device_index):
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(device_index):
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
    except OSError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons)}


def _instance():
    import workloads
    return workloads.standard(WORKLOAD, 0)


# ------------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): runs in a child process, single-threaded BLAS
# ------------------------------------------------------------------------------------------

def _oracle_child(shots_per_p: int, seed: int, offset: int, out_path: str = ""):
    """Decodes shots offset .. offset + shots_per_p - 1 at every p of the sweep with the oracle;
    with out_path, also saves every shot's status, iterations and packed correction there."""
    import numpy as np
    import workloads
    from oracle import lead as olead, philox, tanner
    inst = workloads.standard(WORKLOAD, 0)
    oc = tanner.from_instance(inst)
    from oracle import local
    local.tables(oc.sides[0].RA, oc.sides[0].RB)          # p-independent tables, outside the timing
    wall0 = time.time()
    t0 = time.perf_counter()
    fails = 0
    saved = {}
    for pi, p in enumerate(P_SWEEP):
        x, _ = philox.sample_errors(philox.NOISE_X, p, seed, offset + np.arange(shots_per_p), oc.n)
        syn = philox.syndromes(oc.HZ, x)
        corr, st, it, _ = olead.decode(oc, 0, syn, p)
        fails += int((olead.check(oc, 0, x, corr) != 0).sum())
        if out_path:
            saved[f"corr{pi}"] = philox.pack_bits(corr, (oc.n + 31) // 32)
            saved[f"status{pi}"] = st
            saved[f"iters{pi}"] = it
    dt = time.perf_counter() - t0
    if out_path:
        np.savez(out_path, **saved)
    print(json.dumps({"shots": shots_per_p * len(P_SWEEP), "seconds": dt, "failures": fails,
                      "wall_start": wall0, "wall_end": time.time()}))


def _host_cores() -> int:
    """Host cores this process may run on, at most 64: each oracle process holds its own
    tables, about 100 MB."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(n, 64))


def _run_oracle(shots_per_p: int, seed: int = 0, offset: int = 0, procs: int = 1, out_dir: str = ""):
    """Runs `procs` single-threaded oracle children at once, child i on shot indices
    offset + i * shots_per_p + [0, shots_per_p) at every p. Throughput is measured over the wall
    window from the first child's start of decoding to the last child's end (table setup and
    interpreter start-up excluded); `per_core` is the mean of the children's own rates, i.e. one
    core's rate while all of them are busy. With out_dir, child i saves its outputs as
    out_dir/oracle_<i>.npz."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    children = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-child", str(shots_per_p),
                                  str(seed), str(offset + i * shots_per_p)] +
                                 ([os.path.join(out_dir, f"oracle_{i}.npz")] if out_dir else []),
                                 stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT)
                for i in range(procs)]
    outs = []
    for c in children:
        out, err = c.communicate()
        if c.returncode != 0:
            raise RuntimeError("oracle child failed: " + err[-2000:])
        outs.append(json.loads(out.strip().splitlines()[-1]))
    shots = sum(o["shots"] for o in outs)
    return {"shots": shots, "failures": sum(o["failures"] for o in outs), "procs": procs,
            "seconds": max(o["wall_end"] for o in outs) - min(o["wall_start"] for o in outs),
            "per_core": sum(o["shots"] / o["seconds"] for o in outs) / procs}


# ------------------------------------------------------------------------------------------

def _serving(lead, rates, n: int, code_psl7, unloaded_n: int = 2000):
    """Latency and throughput of single-syndrome requests on the continuous-batching server:
    Poisson arrivals at each offered rate, 70 % PSL(2,7) / 30 % PSL(2,11), depolarizing p = 0.03
    (both sides decoded); then the unloaded latency: requests 1 ms apart, so each one is alone on
    the device (a batch of one)."""
    import numpy as np
    import workloads
    from paper_2605_17796_gb300 import serving as sv
    code11 = lead.Code.from_instance(workloads.standard("PSL(2,11)", 0)).prepare(code_psl7.info.prepared_device)
    codes = [code_psl7, code11]
    p = 0.03
    srv = lead.Server(codes, [2 * p / 3] * 2, max_batch=256, streams=6, budget_bytes=2 << 30)
    # warm-up: a short trace so every kernel is loaded before the measured ones
    warm_arr, warm_code = sv.poisson_trace(rates[0], 2000, [0.7, 0.3], np.random.default_rng(1))
    warm_rows = [sv.request_rows(c, p, int((warm_code == i).sum()), seed=200 + i) for i, c in enumerate(codes)]
    sv.run_trace(srv, warm_rows, warm_arr, warm_code)
    runs = []
    for k, rate in enumerate(rates):
        rng = np.random.default_rng(k)
        arrival, code_of = sv.poisson_trace(rate, n, [0.7, 0.3], rng)
        rows = [sv.request_rows(c, p, int((code_of == i).sum()), seed=100 + 10 * k + i) for i, c in enumerate(codes)]
        res, _ = sv.run_trace(srv, rows, arrival, code_of)
        runs.append(sv.latency_stats(res, rate))
    # unloaded: evenly spaced requests 1 ms apart
    code_of = np.random.default_rng(7).choice(2, size=unloaded_n, p=[0.7, 0.3]).astype(np.int32)
    arrival = (np.arange(unloaded_n, dtype=np.int64) * 1_000_000)
    rows = [sv.request_rows(c, p, int((code_of == i).sum()), seed=300 + i) for i, c in enumerate(codes)]
    res, _ = sv.run_trace(srv, rows, arrival, code_of)
    unloaded = sv.latency_stats(res, 1000.0)
    unloaded["per_code"] = {name: {"p50_us": float(np.percentile(((res["done_ns"] - res["arrival_ns"]) / 1e3)[res["code"] == i], 50)),
                                   "p99_us": float(np.percentile(((res["done_ns"] - res["arrival_ns"]) / 1e3)[res["code"] == i], 99))}
                            for i, name in enumerate(("PSL(2,7)", "PSL(2,11)"))}
    srv.close()
    # the same traffic at the top rate in bfloat16 storage, the PSL(2,11) kernels autotuned at
    # the serving prior first (fresh code objects: the binary32 ones keep their kernels)
    codes16 = [lead.Code.from_instance(workloads.standard(nm, 0)).prepare(code_psl7.info.prepared_device)
               for nm in ("PSL(2,7)", "PSL(2,11)")]
    for side in (0, 1):
        codes16[1].autotune(side, lead.PREC_BF16, 2 * p / 3, 2048)
    srv = lead.Server(codes16, [2 * p / 3] * 2, max_batch=256, streams=6, budget_bytes=2 << 30,
                      precision=lead.PREC_BF16)
    sv.run_trace(srv, warm_rows, warm_arr, warm_code)
    bf16_runs = []
    for k, rate in enumerate(rates):
        if rate < max(rates):
            continue
        rng = np.random.default_rng(k)
        arrival, code_of = sv.poisson_trace(rate, n, [0.7, 0.3], rng)
        rows = [sv.request_rows(c, p, int((code_of == i).sum()), seed=100 + 10 * k + i) for i, c in enumerate(codes16)]
        res, _ = sv.run_trace(srv, rows, arrival, code_of)
        bf16_runs.append(sv.latency_stats(res, rate))
    srv.close()
    return {"runs": runs, "unloaded": unloaded, "mix": "70% PSL(2,7) / 30% PSL(2,11)",
            "noise": "depolarizing p=0.03, both sides", "max_batch": 256, "streams": 6,
            "bf16_tuned_top_rate": bf16_runs}


def _prior_local(lead, code, tc_peak_tflops: float, shots: int = 1 << 15, p: float = 0.02):
    """Phase 1 under per-qubit priors (p_i uniform on [p/2, 3p/2]) on the sweep's code: vertex
    items per second of lead_local_estimate_priors (prior LLRs, local posteriors, merge) with the
    tensor-core kernel and with the CUDA-core kernel, CUDA events around each call. The tensor
    cores compute 2 terms x 2 x (Delta 2^kB) x NK multiply-adds per item for each of the two
    contractions (K1 = 48, NK = 512 on this code)."""
    import torch
    info = code.info
    sz = torch.zeros((shots, info.words_m[0]), dtype=torch.int32, device="cuda")
    ex = torch.zeros((shots, info.words_n), dtype=torch.int32, device="cuda")
    code.sample(lead.NOISE_X, p, shots, 11, 0, err_x=ex, syn_z=sz)
    g = torch.Generator(device="cuda").manual_seed(3)
    prior = torch.rand((shots, info.n), generator=g, device="cuda") * p + 0.5 * p
    lam = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    o = lead.opts(side=0, p=p)
    ws = torch.zeros(code.priors_workspace_bytes(o, shots) // 4 + 64, dtype=torch.int32, device="cuda")
    out = {"shots": shots, "p_range": [0.5 * p, 1.5 * p]}
    for name, simt in (("tensor_cores", "0"), ("cuda_cores", "1")):
        os.environ["LEAD_PRIOR_SIMT"] = simt
        code.local_estimate_priors(o, sz, shots, prior, lam, workspace=ws)       # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            code.local_estimate_priors(o, sz, shots, prior, lam, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        out[name] = {"items_per_s": shots * info.order / (ms / 1e3), "shots_per_s": shots / (ms / 1e3)}
    os.environ.pop("LEAD_PRIOR_SIMT", None)
    flops = 2 * 2 * 2 * (info.delta * 8) * 512            # two contractions, two terms, 2 flops per MAC
    tc = out["tensor_cores"]["items_per_s"] * flops / 1e12
    out["tensor_contraction"] = {"flops_per_item": flops, "achieved_tflops": tc, "peak_tflops": tc_peak_tflops,
                                 "frac": tc / tc_peak_tflops,
                                 "note": "whole call timed (prior LLRs, CUDA-core log-sums, least-cost search, merge)"}
    return out


def _compare_with_oracle(lead, code, pipe, decode, out_dir: str, procs: int, shots_per_p: int):
    """The GPU's outputs for the shots the oracle children decoded (seed 0, shots
    0 .. procs * shots_per_p - 1 at every p): the number of shots whose status, iteration count
    or correction differs from the oracle's."""
    import numpy as np
    info = code.info
    n_sh = procs * shots_per_p
    words = (info.n + 31) // 32
    mism = 0
    for pi, p in enumerate(P_SWEEP):
        code.sample(lead.NOISE_X, p, n_sh, 0, 0, err_x=pipe.err[0], syn_z=pipe.syn[0])
        decode(lead.opts(side=0, p=p), pipe.syn[0], n_sh, pipe.corr[0], pipe.status[0], pipe.iters[0],
               workspace=pipe.workspace)
        corr = pipe.corr[0][:n_sh].cpu().numpy().view(np.uint32)
        st = pipe.status[0][:n_sh].cpu().numpy()
        it = pipe.iters[0][:n_sh].cpu().numpy()
        for i in range(procs):
            z = np.load(os.path.join(out_dir, f"oracle_{i}.npz"))
            sl = slice(i * shots_per_p, (i + 1) * shots_per_p)
            bad = ((z[f"status{pi}"] != st[sl]) | (z[f"iters{pi}"] != it[sl]) |
                   (z[f"corr{pi}"] != corr[sl, :words]).any(axis=1) | (corr[sl, words:] != 0).any(axis=1))
            mism += int(bad.sum())
    return mism, n_sh * len(P_SWEEP)


def _minsum_baseline(lead, pipe, sink, shots_per_p: int):
    """The plain global min-sum baseline (use_lead = 0: channel prior, same iteration cap) on the
    same shots as the first timed LEAD step: per p, decode shots/s (CUDA events around the decode
    calls), logical error rate with its Wilson interval and mean iterations."""
    import torch
    from paper_2605_17796_gb300 import replicas
    out = {}
    tot_ms, tot = 0.0, 0
    for pi, p in enumerate(P_SWEEP):
        off = replicas.shot_offset(0, 0, 1, pi, len(P_SWEEP), shots_per_p)
        sink[0] = []
        r = pipe.run(lead.NOISE_X, p, shots_per_p, seed=0, offset=off, use_lead=False)
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1, _ in sink[0])
        sink[0] = None
        tot_ms += ms
        tot += shots_per_p
        out[f"{p:.2f}"] = {"decode_shots_per_s": shots_per_p / (ms / 1e3), "ler": r.failures / shots_per_p,
                           "ler_ci95": wilson95(r.failures, shots_per_p), "mean_iters": r.iters_sum / shots_per_p}
    return {"shots_per_p": shots_per_p, "decode_shots_per_s": tot / (tot_ms / 1e3), "per_p": out}


from paper_2605_17796_gb300.stats import wilson95  # noqa: E402


MODES = {"fp32": 0, "bf16": 1, "fp16": 2}


def _local_estimation(lead, code, pipe, hbm_peak: float, shots: int):
    """lead_local_estimate (Phases 1-2 alone: class/pair tables, per-(shot, qubit) lookups)
    on the sweep's syndromes, per precision mode: shots/s and algorithmic HBM bytes per second
    (syndromes read + LLRs written) over CUDA events around each call."""
    import torch
    info = code.info
    stream = torch.cuda.current_stream()
    out = {}
    syn_bytes = info.words_m[0] * 4
    for name, prec in MODES.items():
        esize = 4 if prec == 0 else 2
        llr = torch.empty((shots, info.n), dtype=torch.float32 if esize == 4 else torch.int16, device="cuda")
        tot_ms, tot_shots = 0.0, 0
        for p in P_SWEEP:
            code.sample(lead.NOISE_X, p, shots, 3, 0, err_x=pipe.err[0], syn_z=pipe.syn[0])
            o = lead.opts(side=0, p=p, precision=prec)
            code.local_estimate(o, pipe.syn[0], shots, llr, pipe.workspace)        # warm-up
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                code.local_estimate(o, pipe.syn[0], shots, llr, pipe.workspace)
            e1.record(stream)
            torch.cuda.synchronize()
            tot_ms += e0.elapsed_time(e1)
            tot_shots += 3 * shots
        del llr
        gbs = tot_shots * (syn_bytes + info.n * esize) / (tot_ms / 1e3) / 1e9
        out[name] = {"shots_per_s": tot_shots / (tot_ms / 1e3), "algorithmic_gbs": gbs,
                     "frac_of_hbm": gbs / hbm_peak, "bytes_per_shot": syn_bytes + info.n * esize}
    return out


def _kept(report: str) -> str:
    """The candidate lead_code_autotune kept, from its report."""
    for line in report.splitlines():
        if "<- kept" in line:
            return line.replace("<- kept", "").strip()
    return ""


def _precision_modes(lead, pipe, shots: int, p: float = 0.05, tune_shots: int = 65536):
    """Decode throughput and logical error rate (Wilson 95 % interval) of each storage mode on
    the same shots at one p. Each mode's min-sum kernel is first autotuned (lead_code_autotune:
    its register cap chosen by timing, outputs unchanged) on sampled shots at the same p."""
    import torch
    out = {}
    for name, prec in MODES.items():
        kept = _kept(pipe.code.autotune(0, prec, p, tune_shots))
        pipe.run(lead.NOISE_X, p, min(shots, pipe.chunk), seed=5, offset=0, precision=prec)   # warm-up
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = pipe.run(lead.NOISE_X, p, shots, seed=5, offset=0, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"shots_per_s": shots / (ms / 1e3), "ler": r.failures / shots,
                     "ler_ci95": wilson95(r.failures, shots), "mean_iters": r.iters_sum / shots,
                     "kernel": kept}
    return out


def _batch(lead, dev, scale: float = 0.1, reps: int = 1):
    """The multi-code batch (SL(2,3) / PSL(2,7) / PSL(2,11) with 10^4 / 2x10^5 / 10^6 shots times
    `scale`, depolarizing p = 0.04, both sides): eager on one stream with the default kernels,
    then kernels and plan autotuned and the batch replayed as one CUDA graph."""
    import workloads
    from paper_2605_17796_gb300 import batch as mb
    names = ("SL(2,3)", "PSL(2,7)", "PSL(2,11)")
    codes = [lead.Code.from_instance(workloads.standard(n, 0)).prepare(dev) for n in names]
    entries = [mb.Entry(codes[0], int(1e4 * scale), seed=1), mb.Entry(codes[1], int(2e5 * scale), seed=2),
               mb.Entry(codes[2], int(1e6 * scale), seed=3)]
    eager_ms, eager_summary = mb.eager_run(entries, reps)
    best, timings = mb.autotune(entries, reps=reps)
    ms = best.time_replays(reps)
    rep = mb.run_report(names, entries, best, timings, ms, eager_ms, eager_summary, reps)
    rep["scale"] = scale
    del best
    return rep


def _iterated_lead(lead, pipe, shots: int, ps=(0.02, 0.03), rounds=(1, 2, 3)):
    """Iterated LEAD (an extension: further rounds on the unconverged shots, the last global
    posterior as per-qubit prior): logical error rate, mean global iterations summed over rounds,
    and decode throughput per (p, rounds) on the same shots."""
    import torch
    out = []
    for p in ps:
        for R in rounds:
            pipe.run(lead.NOISE_X, p, min(shots, 4096), seed=9, offset=0, rounds=R)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            r = pipe.run(lead.NOISE_X, p, shots, seed=9, offset=0, rounds=R)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out.append({"p": p, "rounds": R, "shots_per_s": shots / (ms / 1e3), "ler": r.failures / shots,
                        "ler_ci95": wilson95(r.failures, shots), "mean_iters": r.iters_sum / shots,
                        "not_converged": r.not_converged / shots})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--shots-per-p", type=int, default=1_000_000)
    ap.add_argument("--chunk", type=int, default=1 << 20)
    ap.add_argument("--oracle-shots-per-p", type=int, default=3,
                    help="reference arm: oracle shots per p per process and step")
    ap.add_argument("--baseline-shots-per-p", type=int, default=120,
                    help="cpu_baseline leg: oracle shots per p per process (a little over 30 s of decoding)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-child", nargs="+")
    ap.add_argument("--serving-rates", type=float, nargs="+", default=[1e5, 3e5, 1e6])
    ap.add_argument("--serving-requests", type=int, default=30000)
    ap.add_argument("--minsum-shots-per-p", type=int, default=1_000_000)
    ap.add_argument("--no-minsum", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--precision-shots", type=int, default=1_000_000)
    ap.add_argument("--no-modes", action="store_true")
    ap.add_argument("--iterated-shots", type=int, default=1 << 18)
    ap.add_argument("--batch-scale", type=float, default=0.1)
    ap.add_argument("--no-batch", action="store_true")
    args = ap.parse_args()

    if args.oracle_child:
        a = args.oracle_child
        _oracle_child(int(a[0]), int(a[1]), int(a[2]), a[3] if len(a) > 3 else "")
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        per_step = []
        procs = _host_cores()
        for s in range(args.warmup + args.steps):
            r = _run_oracle(args.oracle_shots_per_p, 0, s * procs * args.oracle_shots_per_p, procs)
            if s >= args.warmup:
                per_step.append(r)
        shots = sum(r["shots"] for r in per_step)
        secs = sum(r["seconds"] for r in per_step)
        value = shots / secs
        per_core = sum(r["per_core"] for r in per_step) / len(per_step)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32",
                "data": "synthetic",
                "config": {"workload": f"{WORKLOAD} Delta=6 quantum Tanner code, X noise p=0.01..0.10, "
                                       f"oracle sample of {procs} x {args.oracle_shots_per_p} shots per p per step",
                           "max_iter": 32, "alpha": 1.0},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                                 "per_core": per_core,
                                 "sample": f"{procs} single-threaded processes x {args.oracle_shots_per_p} "
                                           f"shots per p x 10 p values per step"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    dev = local_rank

    from paper_2605_17796_gb300 import lead, replicas
    from paper_2605_17796_gb300.pipeline import Pipeline

    inst = _instance()
    code = lead.Code.from_instance(inst).prepare(dev)
    info = code.info
    pipe = Pipeline(code, args.chunk, dev)
    stream = torch.cuda.current_stream()

    # ---- per-kernel CUDA-event timing of the decode call inside the timed region -------------
    decode_events = []
    orig_decode = code.decode
    sink = [None]          # the list that records (start, end, shots) of each decode call, or None

    def timed_decode(*a, **k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        orig_decode(*a, **k)
        e1.record(stream)
        if sink[0] is not None:
            sink[0].append((e0, e1, a[2]))

    code.decode = timed_decode

    results = {}

    def step(step_idx):
        out = []
        for pi, p in enumerate(P_SWEEP):
            off = replicas.shot_offset(step_idx, rank, world, pi, len(P_SWEEP), args.shots_per_p)
            out.append(pipe.run(lead.NOISE_X, p, args.shots_per_p, seed=0, offset=off))
        return out

    # the binary32 kernel's launch shape, chosen by timing at the sweep's priors up to 0.05 (from
    # there on every shot runs the 32 iterations); each p of the sweep uses the shape tuned
    # nearest to it (outputs do not depend on it)
    tuned = {f"{tp:.2f}": _kept(code.autotune(0, lead.PREC_FP32, tp, 65536)) for tp in TUNE_P}
    for w in range(args.warmup):
        step(10_000 + w)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk_dir = tempfile.mkdtemp(prefix="lead_bench_")
    clk_path = os.path.join(clk_dir, f"clocks_rank{rank}.csv")
    sampler = _clock_sampler(clk_path) if local_rank == 0 else None
    time.sleep(0.3)
    sink[0] = decode_events
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sweeps = [step(s) for s in range(args.steps)]
    sweep = sweeps[-1]
    ev1.record(stream)
    torch.cuda.synchronize()
    sink[0] = None
    if world > 1:
        torch.distributed.barrier()
    if sampler:
        sampler.terminate()
        sampler.wait()
    elapsed_ms = replicas.max_over_ranks(ev0.elapsed_time(ev1), world, device="cuda")
    # failure and iteration counts of the last timed sweep, over all ranks
    counts = replicas.sum_over_ranks([r.failures for r in sweep] + [r.iters_sum for r in sweep] +
                                     [r.shots for r in sweep], world, device="cuda")
    n_p = len(P_SWEEP)
    sweep_fail, sweep_iters, sweep_shots = counts[:n_p], counts[n_p:2 * n_p], counts[2 * n_p:]
    total_shots = args.steps * len(P_SWEEP) * args.shots_per_p * world
    value = total_shots / (elapsed_ms / 1e3)

    # decode kernel time inside the timed region
    dec_ms = sum(e0.elapsed_time(e1) for e0, e1, _ in decode_events)
    chunks_per_p = -(-args.shots_per_p // args.chunk)
    launches_per_chunk = 5          # sample, local table, class tables, min-sum decode, check
    gpu_launches = args.steps * len(P_SWEEP) * chunks_per_p * launches_per_chunk

    # ---- e2e: host syndromes and errors in pinned memory -> decode -> corrections back ------
    e2e = None
    if rank == 0:
        e2e_shots = min(args.chunk, 1 << 18)
        hsyn, herr = {}, {}
        for p in P_SWEEP:
            pipe.code.sample(lead.NOISE_X, p, e2e_shots, 7, 0, err_x=pipe.err[0], syn_z=pipe.syn[0])
            hsyn[p] = pipe.syn[0][:e2e_shots].cpu().pin_memory()
            herr[p] = pipe.err[0][:e2e_shots].cpu().pin_memory()
        # two streams take alternate p values with their own rows of the pipeline's buffers, own
        # workspace and own pinned result buffers, so one p's copies overlap the other's decode
        streams = [stream, torch.cuda.Stream()]
        wss = [pipe.workspace, torch.zeros_like(pipe.workspace)]
        hout = [{"corr": torch.empty((e2e_shots, info.words_n), dtype=torch.int32).pin_memory(),
                 "fail": torch.empty(e2e_shots, dtype=torch.uint8).pin_memory(),
                 "stat": torch.empty(e2e_shots, dtype=torch.uint8).pin_memory()} for _ in range(2)]

        def e2e_step():
            streams[1].wait_stream(stream)       # after whatever the step follows (its start event)
            for k, p in enumerate(P_SWEEP):
                b = k % 2
                rows = slice(b * e2e_shots, (b + 1) * e2e_shots)
                st = streams[b]
                with torch.cuda.stream(st):
                    syn, err = pipe.syn[0][rows], pipe.err[0][rows]
                    corr, sta, its, fail = pipe.corr[0][rows], pipe.status[0][rows], pipe.iters[0][rows], pipe.fail[0][rows]
                    syn.copy_(hsyn[p], non_blocking=True)
                    err.copy_(herr[p], non_blocking=True)
                    o = lead.opts(side=0, p=p)
                    orig_decode(o, syn, e2e_shots, corr, sta, its, workspace=wss[b], stream=st)
                    code.check(0, err, corr, e2e_shots, fail, stream=st)
                    hout[b]["corr"].copy_(corr, non_blocking=True)
                    hout[b]["fail"].copy_(fail, non_blocking=True)
                    hout[b]["stat"].copy_(sta, non_blocking=True)
            stream.wait_stream(streams[1])
        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        reps = max(1, args.steps // 2)
        a0.record(stream)
        for _ in range(reps):
            e2e_step()
        a1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = a0.elapsed_time(a1)
        bi = e2e_shots * (info.words_m[0] + info.words_n) * 4 * len(P_SWEEP)
        bo = e2e_shots * (info.words_n * 4 + 2) * len(P_SWEEP)
        e2e = {"value": reps * e2e_shots * len(P_SWEEP) / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
               "shots_per_step": e2e_shots * len(P_SWEEP)}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (the fused LEAD min-sum decode) ---------------------
    peaks, peak_kind = _peaks()
    iters_total = sum(r.iters_sum for sw in sweeps for r in sw)     # min-sum shot-iterations
    H = code.check_matrix(0)
    E = int(H.sum())
    # algorithmic work of flooding min-sum per edge and iteration: v2c subtract, |.|, two
    # compares (min1/min2), sign parity, posterior add = 6 ops. Three of them (the compares and
    # the parity bit operation) issue on the ALU pipe, 64 lanes per SM (16 per sub-partition);
    # the other three on the FMA pipe, 128 lanes per SM. The ALU pipe binds: 64/3 edges per
    # SM-cycle = 128 algorithmic ops per SM-cycle.
    ops = 6.0 * E * iters_total
    clock_mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = 152 * 128 * clock_mhz * 1e6 / 1e12         # Tops/s
    achieved = ops / (dec_ms / 1e3) / 1e12 if dec_ms > 0 else None
    roofline = {"kernel": "lead_bp_jit (fused local estimation lookup + merge + min-sum)", "bound": "alu",
                "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                "frac": (achieved / alu_peak) if achieved else None, "traffic": None,
                "peak_source": (f"derived: 152 SMs x {clock_mhz:.0f} MHz x 128 ops per SM-cycle; 6 ops per edge "
                                f"and iteration, 3 on the ALU pipe (64 lanes per SM, binding: 64/3 edges per "
                                f"SM-cycle) and 3 on the FMA pipe (128 lanes per SM)"),
                "work_per_unit": f"6 ops x {E} edges per shot-iteration; {iters_total} shot-iterations",
                "decode_ms_in_timed_region": dec_ms}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        procs = _host_cores()
        out_dir = tempfile.mkdtemp(prefix="lead_oracle_")
        r = _run_oracle(args.baseline_shots_per_p, 0, 0, procs, out_dir=out_dir)
        mism, compared = _compare_with_oracle(lead, code, pipe, orig_decode, out_dir, procs, args.baseline_shots_per_p)
        cpu = {"value": r["shots"] / r["seconds"], "unit": UNIT, "cores": procs, "kind": "oracle",
               "per_core": r["per_core"],
               "sample": f"{procs} single-threaded numpy processes x {args.baseline_shots_per_p} shots per p "
                         f"x 10 p values on disjoint shots ({r['shots']} shots, {r['seconds']:.1f} s wall)",
               "mismatches": mism, "compared_shots": compared,
               "compared": "status, iterations and correction of every oracle shot against the GPU's"}

    minsum = None
    if not args.no_minsum and world == 1:
        minsum = _minsum_baseline(lead, pipe, sink, args.minsum_shots_per_p)

    local_est = precision = precision11 = iterated = prior_local = None
    if not args.no_modes and world == 1:
        local_est = _local_estimation(lead, code, pipe, peaks["hbm_gbs"], min(args.chunk, 1 << 20))
        prior_local = _prior_local(lead, code, peaks.get("bf16_tflops", 1900.0))
        precision = _precision_modes(lead, pipe, args.precision_shots)
        import workloads
        code11 = lead.Code.from_instance(workloads.standard("PSL(2,11)", 0)).prepare(dev)
        pipe11 = Pipeline(code11, 1 << 15, dev)
        precision11 = _precision_modes(lead, pipe11, 1 << 16, p=PSL11_P, tune_shots=8192)
        del pipe11, code11
        iterated = _iterated_lead(lead, pipe, min(args.iterated_shots, args.chunk))

    serving = None
    if not args.no_serving and world == 1:
        serving = _serving(lead, args.serving_rates, args.serving_requests, code)

    batch = None
    if not args.no_batch and world == 1:
        batch = _batch(lead, dev, args.batch_scale)

    clocks = _clock_summary(clk_path, dev)
    ler = {f"{p:.2f}": f / n for p, f, n in zip(P_SWEEP, sweep_fail, sweep_shots)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} Delta=6 quantum Tanner code (n={info.n}, k={info.k}), "
                                   f"code-capacity X noise p=0.01..0.10, {args.shots_per_p} shots per p",
                       "shots_per_step": len(P_SWEEP) * args.shots_per_p * world, "max_iter": 32,
                       "alpha": 1.0, "decoder": "LEAD (exact local estimation + merge + min-sum)",
                       "l2": "inputs larger than L2 (2^20-shot chunks, 400 MB of errors)",
                       "parallelism": f"replicas x{world}", "min_sum_kernel_by_tuning_p": tuned},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
            "minsum_baseline": minsum,
            "local_estimation": local_est, "prior_local": prior_local,
            "precision_modes": ({"p": 0.05, "shots": args.precision_shots, "modes": precision}
                                if precision else None),
            "precision_modes_psl11": ({"code": "PSL(2,11) (n=11880)", "p": PSL11_P, "shots": 1 << 16,
                                       "modes": precision11} if precision11 else None),
            "iterated_lead": ({"shots": min(args.iterated_shots, args.chunk), "runs": iterated}
                              if iterated else None),
            "serving": serving,
            "batch": batch,
            "clocks": clocks, "ler": ler,
            "mean_iters": {f"{p:.2f}": i / n for p, i, n in zip(P_SWEEP, sweep_iters, sweep_shots)}}
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
