"""Parity on the benchmark's own workload, through the C ABI.

The workload: the seeded PSL(2,7) code (|G| = 168, Delta = 6, n = 3024), side 0 (code-capacity
X noise), LEAD in binary32 with alpha = 1 and at most 32 global min-sum iterations, at every p
of the sweep 0.01 ... 0.10. The shots are the benchmark's: seed 0 and the absolute shot indices
of its first timed step (replicas.shot_offset(0, 0, 1, p index, 10, 10^6)).

* 1 000 shots per p (10 000 in all): corrections, statuses, iteration counts, final posteriors
  and the Sec. IV-A check flags equal the oracle's, bit for bit;
* the benchmark's launch configuration (one decode call over the 10^6 shots of one p, without
  posterior output): sampled rows (the first 64, 64 spread over the call, the last 8) equal the
  oracle's at p = 0.03, 0.05 and 0.08;
* the binary32 decision track against the oracle's FP64 track (prior_f64 and min-sum in
  binary64, same rules), on 3 400 benchmark shots at each of p = 0.01, 0.03 and 0.05: the shots
  whose failure verdict differs, and those converged on both tracks with different corrections,
  are counted and stay under stated bounds.

The oracle runs in a process pool (spawn) while the GPU decodes.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle_workers as ow  # noqa: E402

P_SWEEP = [round(0.01 * i, 2) for i in range(1, 11)]
SHOTS_PER_P = 1000
BENCH_SHOTS_PER_P = 1_000_000
JOB = 50
# binary32 against the FP64 track: the p values compared, and the fractions of shots allowed a
# different failure verdict, and a different correction among shots converged on both tracks
F64_P = (0.01, 0.03, 0.05)
F64_SHOTS_PER_P = 3400        # 10 200 shots over the three p values
VERDICT_BOUND = 0.02
CONVERGED_BOUND = 0.01


def _offset(pi):
    from paper_2605_17796_gb300 import replicas
    return replicas.shot_offset(0, 0, 1, pi, len(P_SWEEP), BENCH_SHOTS_PER_P)


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2605_17796_gb300 import lead
    return lead


@pytest.fixture(scope="module")
def pool():
    n = max(1, min(32, os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
        yield ex


@pytest.fixture(scope="module")
def code(L):
    import workloads
    return L.Code.from_instance(workloads.standard("PSL(2,7)", 0)).prepare(0)


def _gpu_decode(L, code, p, shots, offset, with_post=True):
    info = code.info
    ex = torch.zeros((shots, info.words_n), dtype=torch.int32, device="cuda")
    sz = torch.zeros((shots, info.words_m[0]), dtype=torch.int32, device="cuda")
    code.sample(L.NOISE_X, p, shots, 0, offset, err_x=ex, syn_z=sz)
    o = L.opts(side=0, p=p)
    ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
    corr = torch.full((shots, info.words_n), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    it = torch.full((shots,), -1, dtype=torch.int32, device="cuda")
    post = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda") if with_post else None
    code.decode(o, sz, shots, corr, st, it, post, workspace=ws)
    fail = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    code.check(0, ex, corr, shots, fail)
    torch.cuda.synchronize()
    return corr, st, it, post, fail


def _bits(t, rows, n):
    from oracle import philox
    return philox.unpack_bits(t[rows].cpu().numpy().view(np.uint32), n)


def _gather(futs):
    parts = [f.result() for f in futs]
    return {k: np.concatenate([r[k] for r in parts]) for k in parts[0]}


def test_headline_sweep_every_p(L, code, pool):
    n = code.info.n
    jobs = {}
    for pi, p in enumerate(P_SWEEP):
        idx = _offset(pi) + np.arange(SHOTS_PER_P)
        jobs[p] = [pool.submit(ow.decode_shots, "PSL(2,7)", 0, p, 0, idx[i:i + JOB]) for i in range(0, SHOTS_PER_P, JOB)]
    for pi, p in enumerate(P_SWEEP):
        corr, st, it, post, fail = _gpu_decode(L, code, p, SHOTS_PER_P, _offset(pi))
        want = _gather(jobs[p])
        rows = torch.arange(SHOTS_PER_P, device="cuda")
        assert (st.cpu().numpy() == want["status"]).all(), p
        assert (it.cpu().numpy() == want["iters"]).all(), p
        assert (_bits(corr, rows, n) == want["corr"]).all(), p
        assert (post.cpu().numpy().view(np.uint32) == want["post"].view(np.uint32)).all(), p
        assert (fail.cpu().numpy() == want["fail"]).all(), p


@pytest.mark.parametrize("p", [0.03, 0.05, 0.08])
def test_headline_full_call_sampled_rows(L, code, pool, p):
    pi = P_SWEEP.index(p)
    off = _offset(pi)
    rng = np.random.default_rng(int(p * 1000))
    rows = np.unique(np.concatenate([np.arange(64), rng.integers(64, BENCH_SHOTS_PER_P - 8, 64),
                                     np.arange(BENCH_SHOTS_PER_P - 8, BENCH_SHOTS_PER_P)]))
    futs = [pool.submit(ow.decode_shots, "PSL(2,7)", 0, p, 0, off + rows[i:i + JOB]) for i in range(0, len(rows), JOB)]
    corr, st, it, _, fail = _gpu_decode(L, code, p, BENCH_SHOTS_PER_P, off, with_post=False)
    want = _gather(futs)
    r = torch.from_numpy(rows).cuda()
    assert (st[r].cpu().numpy() == want["status"]).all()
    assert (it[r].cpu().numpy() == want["iters"]).all()
    assert (_bits(corr, r, code.info.n) == want["corr"]).all()
    assert (fail[r].cpu().numpy() == want["fail"]).all()


def test_binary32_track_against_fp64_track(L, code, pool):
    """How often binary32 rounding changes the outcome: the GPU (equal to the oracle's binary32
    track, above) against the oracle's FP64 track on 3 400 benchmark shots per p. Min-sum that
    does not converge wanders, and its last decision depends on every rounding, so two counts are
    held: shots whose failure verdict (Sec. IV-A) differs, and shots that converged on both tracks
    with different corrections."""
    n = code.info.n
    for p in F64_P:
        pi = P_SWEEP.index(p)
        m = F64_SHOTS_PER_P
        idx = _offset(pi) + np.arange(m)
        futs = [pool.submit(ow.decode_shots, "PSL(2,7)", 0, p, 0, idx[i:i + JOB], True, "f64")
                for i in range(0, m, JOB)]
        corr, st, it, _, fail = _gpu_decode(L, code, p, m, _offset(pi), with_post=False)
        want = _gather(futs)
        st = st.cpu().numpy()
        both = (st == L.ST_CONVERGED) & (want["status"] == L.ST_CONVERGED)
        diff = (_bits(corr, torch.arange(m, device="cuda"), n) != want["corr"]).any(axis=1)
        verdict = int(((fail.cpu().numpy() != 0) != (want["fail"] != 0)).sum())
        conv_diff = int((diff & both).sum())
        print(f"p={p}: failure verdicts differing from the FP64 track {verdict}/{m}; shots "
              f"converged on both tracks {int(both.sum())}, of them with different corrections {conv_diff}")
        assert verdict <= VERDICT_BOUND * m
        assert conv_diff <= CONVERGED_BOUND * m
