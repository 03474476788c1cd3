"""Multi-code batch in one CUDA-graph launch (kernels and plan autotuned): every entry's
corrections, statuses and failure flags equal those of the same entry decoded on its own,
eagerly, and sampled rows of every code equal the oracle's decode of the same shots; replays
are repeatable."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_graph_batch_equals_separate_runs():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2605_17796_gb300 import lead
    from paper_2605_17796_gb300.batch import Entry, MultiCodeBatch, autotune

    codes = [lead.Code.from_instance(workloads.standard(n, 0)).prepare(0)
             for n in ("SL(2,3)", "PSL(2,7)", "PSL(2,11)")]
    entries = [Entry(codes[0], 1000, seed=1), Entry(codes[1], 700, seed=2), Entry(codes[2], 120, seed=3)]
    batch, timings = autotune(entries, reps=1)
    assert len(timings) == 6
    batch.replay()
    torch.cuda.synchronize()
    got = [{k: [t.clone() for t in b[k]] for k in ("corr", "status", "iters", "fail")} for b in batch.buf]
    batch.replay()
    torch.cuda.synchronize()
    for g, b in zip(got, batch.buf):
        for k in g:
            for s in (0, 1):
                assert torch.equal(g[k][s], b[k][s])
    for i, e in enumerate(entries):
        solo = MultiCodeBatch([e], plan=[(0, 1)])
        solo.issue()
        torch.cuda.synchronize()
        for k in ("corr", "status", "iters", "fail"):
            for s in (0, 1):
                assert torch.equal(got[i][k][s], solo.buf[0][k][s]), (i, k, s)
    # sampled rows of every code against the oracle (depolarizing p = 0.04: each side decoded
    # with prior 2p/3 from the shot's X or Z part)
    from oracle import lead as olead, philox, tanner
    for i, (e, name) in enumerate(zip(entries, ("SL(2,3)", "PSL(2,7)", "PSL(2,11)"))):
        oc = tanner.from_instance(workloads.standard(name, 0))
        rows = np.array([0, 5, 77] if name != "PSL(2,11)" else [0, 41])
        x, z = philox.sample_errors(philox.NOISE_DEPOL, e.p, e.seed, rows, oc.n)
        for s, err in ((0, x), (1, z)):
            wc, wst, wit, _ = olead.decode(oc, s, philox.syndromes(oc.sides[s].H, err), 2 * e.p / 3)
            words = got[i]["corr"][s][rows].cpu().numpy().view(np.uint32)
            assert (philox.unpack_bits(words, oc.n) == wc).all(), (name, s)
            assert (got[i]["status"][s][rows].cpu().numpy() == wst).all(), (name, s)
            assert (got[i]["iters"][s][rows].cpu().numpy() == wit).all(), (name, s)
