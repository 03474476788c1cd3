"""Local min-sum BP as the Phase-1 LocalDecoder (LEAD_EST_MINSUM) against the oracle.

Bar: the 2^m_l x Delta^2 binary32 table, the local iteration counts and convergence flags are
bit-exact (the same binary32 min-sum and the same binary64 exponential on both sides);
everything downstream (merged LLRs, global min-sum in every storage mode) is bit-exact.
"""
import numpy as np
import pytest

import workloads
from oracle import lead as olead
from oracle import philox, tanner

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2605_17796_gb300 import lead
    return lead


@pytest.fixture(scope="module")
def codes(L):
    out = {}
    for name in ("SL(2,3)", "PSL(2,7)", "PSL(2,11)"):
        inst = workloads.standard(name, 0)
        out[name] = (inst, L.Code.from_instance(inst).prepare(0), tanner.from_instance(inst))
    return out


def _syn(oc, side, shots, p, seed):
    x, z = philox.sample_errors(side, p, seed, np.arange(shots), oc.n)
    e = x if side == 0 else z
    return philox.syndromes(oc.sides[side].H, e)


def _dev_words(bits, words):
    return torch.from_numpy(philox.pack_bits(bits, words).view(np.int32)).cuda()


@pytest.mark.parametrize("name", ["SL(2,3)", "PSL(2,7)"])
@pytest.mark.parametrize("p", [0.01, 0.04, 0.0266667])
def test_minsum_table_bit_exact(codes, L, name, p):
    inst, code, oc = codes[name]
    for side in (0, 1):
        S, nl = 1 << code.info.m_l[side], inst.delta ** 2
        t = torch.zeros(S * nl, dtype=torch.float32, device="cuda")
        it = torch.zeros(S, dtype=torch.int32, device="cuda")
        code.local_table_est(side, p, L.EST_MINSUM, t, it)
        torch.cuda.synchronize()
        q, iters, conv, _ = olead.local_minsum_tables(oc.sides[side].RA, oc.sides[side].RB, p)
        assert (t.cpu().numpy().reshape(q.shape).view(np.uint32) == q.view(np.uint32)).all()
        got = it.cpu().numpy()
        assert ((got & 0xFFFF) == iters).all()
        assert (((got >> 16) & 1).astype(bool) == conv).all()


def test_exact_estimator_reports_one_iteration(codes, L):
    inst, code, oc = codes["PSL(2,7)"]
    S = 1 << code.info.m_l[0]
    t = torch.zeros(S * 36, dtype=torch.float32, device="cuda")
    it = torch.zeros(S, dtype=torch.int32, device="cuda")
    code.local_table_est(0, 0.03, L.EST_EXACT, t, it)
    t2 = torch.zeros_like(t)
    code.local_table(0, 0.03, t2)
    torch.cuda.synchronize()
    assert torch.equal(t, t2)
    assert (it.cpu().numpy() == (1 | 0x10000)).all()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,side,p,shots", [("SL(2,3)", 0, 0.05, 50), ("PSL(2,7)", 0, 0.02, 16),
                                               ("PSL(2,7)", 1, 0.03, 12), ("PSL(2,11)", 0, 0.02, 4)])
def test_decode_with_minsum_estimator(codes, L, precision, name, side, p, shots):
    inst, code, oc = codes[name]
    info = code.info
    syn = _syn(oc, side, shots, p, 21)
    o = L.opts(side=side, p=p, precision=precision, estimator=L.EST_MINSUM)
    ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
    corr = torch.zeros((shots, info.words_n), dtype=torch.int32, device="cuda")
    st = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    its = torch.zeros(shots, dtype=torch.int32, device="cuda")
    post = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    code.decode(o, _dev_words(syn, info.words_m[side]), shots, corr, st, its, post, ws)
    torch.cuda.synchronize()
    wc, wst, wit, wpost = olead.decode(oc, side, syn, p, precision=precision, estimator=olead.EST_MINSUM)
    assert (st.cpu().numpy() == wst).all() and (its.cpu().numpy() == wit).all()
    assert (philox.unpack_bits(corr.cpu().numpy().view(np.uint32), info.n) == wc).all()
    assert (post.cpu().numpy().view(np.uint32) == wpost.view(np.uint32)).all()


@pytest.mark.parametrize("name", ["SL(2,3)", "PSL(2,7)"])
def test_local_estimate_with_minsum_estimator(codes, L, name):
    """The standalone Phases 1-2: class tables for SL(2,3) (few distinct values), the direct
    merge for PSL(2,7) (thousands of distinct min-sum posteriors)."""
    inst, code, oc = codes[name]
    info = code.info
    shots, p = 30, 0.03
    syn = _syn(oc, 0, shots, p, 5)
    o = L.opts(side=0, p=p, estimator=L.EST_MINSUM)
    ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
    llr = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    code.local_estimate(o, _dev_words(syn, info.words_m[0]), shots, llr, ws)
    torch.cuda.synchronize()
    want = olead.prior_f32(oc, 0, syn, p, estimator=olead.EST_MINSUM)
    assert (llr.cpu().numpy().view(np.uint32) == want.view(np.uint32)).all()


def test_unknown_estimator_rejected(codes, L):
    inst, code, oc = codes["SL(2,3)"]
    t = torch.zeros(16 * 16, dtype=torch.float32, device="cuda")
    with pytest.raises(L.LeadError):
        code.local_table_est(0, 0.03, 7, t)
    o = L.opts(side=0, p=0.03, estimator=7)
    ws = torch.zeros(code.workspace_bytes(L.opts(side=0, p=0.03)) // 4 + 64, dtype=torch.int32, device="cuda")
    syn = torch.zeros((2, code.info.words_m[0]), dtype=torch.int32, device="cuda")
    with pytest.raises(L.LeadError):
        code.decode(o, syn, 2, torch.zeros((2, code.info.words_n), dtype=torch.int32, device="cuda"),
                    torch.zeros(2, dtype=torch.uint8, device="cuda"), workspace=ws)
