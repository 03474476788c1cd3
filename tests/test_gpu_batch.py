"""Multi-code batch in one CUDA-graph launch: every entry's corrections, statuses and failure
flags equal those of the same entry decoded on its own, eagerly; replays are repeatable."""
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
