"""The continuous-batching decode server over SL(2,3), PSL(2,7) and PSL(2,11) (the serving
workload mixes the last two): every result equals the batch decode of the same shot, whether the
request was served alone or mixed with other codes' traffic; sampled results of each code equal
the oracle's decode of the same shot (both sides); memory admission."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

NAMES = ("SL(2,3)", "PSL(2,7)", "PSL(2,11)")
ROWS = (100, 150, 60)

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2605_17796_gb300 import lead, serving
    codes = [lead.Code.from_instance(workloads.standard(n, 0)).prepare(0) for n in NAMES]
    p = 0.03
    rows = [serving.request_rows(c, p, k, seed=21 + i) for i, (c, k) in enumerate(zip(codes, ROWS))]
    # reference: one batch decode per code and side, with the same options as the server
    ref = []
    for c, r in zip(codes, rows):
        info = c.info
        n = r.shape[0]
        out = {}
        for side in (0, 1):
            off = 0 if side == 0 else info.words_m[0]
            syn = torch.from_numpy(np.ascontiguousarray(r[:, off:off + info.words_m[side]]).view(np.int32)).cuda()
            o = lead.opts(side=side, p=2 * p / 3)
            ws = torch.zeros(c.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
            corr = torch.zeros((n, info.words_n), dtype=torch.int32, device="cuda")
            st = torch.zeros(n, dtype=torch.uint8, device="cuda")
            c.decode(o, syn, n, corr, st, workspace=ws)
            out[side] = (corr.cpu().numpy().view(np.uint32), st.cpu().numpy())
        ref.append(out)
    torch.cuda.synchronize()
    return lead, serving, codes, rows, ref, p


def _check(res, cor, codes, ref, key_of):
    W = max(c.info.words_n for c in codes)
    for k in range(len(res)):
        c, i = key_of(int(res["id"][k]))
        wn = codes[c].info.words_n
        for side in (0, 1):
            assert res["status"][k][side] == ref[c][side][1][i]
            assert (cor[k, side, :wn] == ref[c][side][0][i]).all()
            assert not cor[k, side, wn:W].any()


def test_mixed_traffic_matches_batch_decode(setup):
    lead, serving, codes, rows, ref, p = setup
    srv = lead.Server(codes, [2 * p / 3] * 3, max_batch=32, streams=3, budget_bytes=256 << 20)
    rng = np.random.default_rng(0)
    n = sum(r.shape[0] for r in rows)
    arrival, code_of = serving.poisson_trace(2e5, n, [1, 1, 1], rng)
    # use every row of every code exactly once
    code_of = np.concatenate([[c] * r.shape[0] for c, r in enumerate(rows)]).astype(np.int32)[rng.permutation(n)]
    res, cor = serving.run_trace(srv, rows, arrival, code_of)
    idx = np.zeros(n, dtype=np.int64)
    for c in range(len(codes)):
        sel = np.nonzero(code_of == c)[0]
        idx[sel] = np.arange(sel.size)
    _check(res, cor, codes, ref, lambda rid: (int(code_of[rid]), int(idx[rid])))
    assert srv.pending() == 0
    srv.close()
    # sampled requests of each code against the oracle (the server decoded row i of code c from
    # the depolarizing shot i of seed 21 + c)
    from oracle import lead as olead, philox, tanner
    for c, name in enumerate(NAMES):
        oc = tanner.from_instance(workloads.standard(name, 0))
        take = np.array([0, 3, 11, 40] if name != "PSL(2,11)" else [0, 9])
        x, z = philox.sample_errors(philox.NOISE_DEPOL, p, 21 + c, take, oc.n)
        sel = np.nonzero(code_of == c)[0]
        for side, e in ((0, x), (1, z)):
            wc, wst, _, _ = olead.decode(oc, side, philox.syndromes(oc.sides[side].H, e), 2 * p / 3)
            for k, i in enumerate(take):
                r = int(np.nonzero(res["id"] == sel[i])[0][0])
                assert res["status"][r][side] == wst[k]
                got = philox.unpack_bits(cor[r:r + 1, side, :codes[c].info.words_n], oc.n)[0]
                assert (got == wc[k]).all()


def test_alone_equals_in_the_mix(setup):
    lead, serving, codes, rows, ref, p = setup
    srv = lead.Server(codes, [2 * p / 3] * 3, max_batch=32, streams=2, budget_bytes=256 << 20)
    for c in range(len(codes)):
        for i in (0, 7, 42):
            srv.submit(c, rows[c][i:i + 1], np.array([1000 * c + i], dtype=np.uint64))
            got = []
            import time
            t_end = time.time() + 30
            while not got and time.time() < t_end:
                r, cr = srv.poll()
                if len(r):
                    got = [(r, cr)]
            r, cr = got[0]
            assert len(r) == 1 and int(r["id"][0]) == 1000 * c + i
            _check(r, cr, codes, ref, lambda rid: (rid // 1000, rid % 1000))
    srv.close()


def test_memory_admission(setup):
    lead, serving, codes, rows, ref, p = setup
    with pytest.raises(lead.LeadError) as e:
        lead.Server(codes, [2 * p / 3] * 3, max_batch=1024, streams=4, budget_bytes=1 << 16)
    assert e.value.rc == -5           # LEAD_EOOM: not even one slot fits the budget
    # a small budget admits fewer slots and still serves every request
    srv = lead.Server(codes, [2 * p / 3] * 3, max_batch=8, streams=4, budget_bytes=400_000)
    arrival, _ = serving.poisson_trace(1e5, 20, [1.0], np.random.default_rng(1))
    res, cor = serving.run_trace(srv, [rows[0][:20], rows[1][:0], rows[2][:0]], arrival,
                                 np.zeros(20, dtype=np.int32))
    _check(res, cor, codes, ref, lambda rid: (0, rid))
    srv.close()


def test_bfloat16_server_matches_bfloat16_batch_decode(setup):
    """A server in bfloat16 storage (its codes autotuned at the serving prior first, so the
    batches run the tuned launch shapes) returns for every request the bfloat16 batch decode of
    the same shot."""
    lead, serving, _, rows, _, p = setup
    codes = [lead.Code.from_instance(workloads.standard(n, 0)).prepare(0) for n in NAMES]
    for c in codes[1:]:
        for side in (0, 1):
            c.autotune(side, lead.PREC_BF16, 2 * p / 3, 512)
    ref = []
    for c, r in zip(codes, rows):
        info = c.info
        n = r.shape[0]
        out = {}
        for side in (0, 1):
            off = 0 if side == 0 else info.words_m[0]
            syn = torch.from_numpy(np.ascontiguousarray(r[:, off:off + info.words_m[side]]).view(np.int32)).cuda()
            o = lead.opts(side=side, p=2 * p / 3, precision=lead.PREC_BF16)
            ws = torch.zeros(c.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
            corr = torch.zeros((n, info.words_n), dtype=torch.int32, device="cuda")
            st = torch.zeros(n, dtype=torch.uint8, device="cuda")
            c.decode(o, syn, n, corr, st, workspace=ws)
            out[side] = (corr.cpu().numpy().view(np.uint32), st.cpu().numpy())
        ref.append(out)
    torch.cuda.synchronize()
    srv = lead.Server(codes, [2 * p / 3] * 3, max_batch=32, streams=3, budget_bytes=256 << 20,
                      precision=lead.PREC_BF16)
    rng = np.random.default_rng(3)
    n = sum(r.shape[0] for r in rows)
    arrival, _ = serving.poisson_trace(2e5, n, [1, 1, 1], rng)
    code_of = np.concatenate([[c] * r.shape[0] for c, r in enumerate(rows)]).astype(np.int32)[rng.permutation(n)]
    res, cor = serving.run_trace(srv, rows, arrival, code_of)
    idx = np.zeros(n, dtype=np.int64)
    for c in range(len(codes)):
        sel = np.nonzero(code_of == c)[0]
        idx[sel] = np.arange(sel.size)
    _check(res, cor, codes, ref, lambda rid: (int(code_of[rid]), int(idx[rid])))
    assert srv.pending() == 0
    srv.close()
    with pytest.raises(lead.LeadError):
        lead.Server(codes, [2 * p / 3] * 3, precision=3)
