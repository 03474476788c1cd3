"""Precision modes (LLR storage in bfloat16 / binary16, binary32 arithmetic) against the oracle.

Bar: the 16-bit local-estimate outputs equal the oracle's binary32 LLRs rounded to the format
(bit patterns); corrections, status, iterations and final posteriors equal the oracle's min-sum
with the same storage rounding, bit for bit. Against the FP64 prior LLRs the stored values stay
within the format's unit roundoff plus the binary32 track's 1e-4: |d| <= 2^-8 |lambda| + 1e-4
(bfloat16, 8 significant bits) and 2^-11 |lambda| + 1e-4 (binary16, 11 bits; the LLRs here are
far above its subnormal range).
"""
import numpy as np
import pytest

import workloads
from oracle import lead as olead
from oracle import philox, tanner

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MODES = [1, 2]        # LEAD_PREC_BF16, LEAD_PREC_FP16
REL = {1: 2.0 ** -8, 2: 2.0 ** -11}


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
    return e, philox.syndromes(oc.sides[side].H, e)


def _dev_words(bits, words):
    return torch.from_numpy(philox.pack_bits(bits, words).view(np.int32)).cuda()


def _as_f32(raw, precision):
    """16-bit patterns (int16 tensor) -> binary32 values."""
    u = raw.cpu().numpy().view(np.uint16)
    if precision == 1:
        return (u.astype(np.uint32) << 16).view(np.float32)
    return u.view(np.float16).astype(np.float32)


@pytest.mark.parametrize("precision", MODES)
@pytest.mark.parametrize("name,side,p,shots", [("SL(2,3)", 0, 0.05, 40), ("PSL(2,7)", 1, 0.03, 16),
                                               ("PSL(2,11)", 0, 0.02, 4)])
def test_local_estimate_16bit(codes, L, precision, name, side, p, shots):
    inst, code, oc = codes[name]
    info = code.info
    e, syn = _syn(oc, side, shots, p, 3)
    o = L.opts(side=side, p=p, precision=precision)
    ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
    out = torch.zeros((shots, info.n), dtype=torch.int16, device="cuda")
    code.local_estimate(o, _dev_words(syn, info.words_m[side]), shots, out, ws)
    torch.cuda.synchronize()
    got = _as_f32(out, precision)
    want32 = olead.prior_f32(oc, side, syn, p)
    want = olead.round_storage(want32, precision)
    assert (got.view(np.uint32) == want.view(np.uint32)).all()
    _, want64 = olead.prior_f64(oc, side, syn, p)
    assert np.all(np.abs(got - want64) <= REL[precision] * np.abs(want64) + 1e-4)


def _decode(L, code, side, syn, p, precision, use_lead=True, alpha=1.0):
    info = code.info
    shots = syn.shape[0]
    o = L.opts(side=side, p=p, alpha=alpha, use_lead=use_lead, precision=precision)
    ws = torch.zeros(max(code.workspace_bytes(o), 256) // 4 + 64, dtype=torch.int32, device="cuda")
    corr = torch.full((shots, info.words_n), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    it = torch.full((shots,), -1, dtype=torch.int32, device="cuda")
    post = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    code.decode(o, _dev_words(syn, info.words_m[side]), shots, corr, st, it, post, ws)
    torch.cuda.synchronize()
    return (philox.unpack_bits(corr.cpu().numpy().view(np.uint32), info.n), st.cpu().numpy(), it.cpu().numpy(),
            post.cpu().numpy())


@pytest.mark.parametrize("precision", MODES)
@pytest.mark.parametrize("name,side,p,shots,use_lead", [
    ("SL(2,3)", 0, 0.04, 60, True), ("SL(2,3)", 1, 0.08, 40, False),
    ("PSL(2,7)", 0, 0.02, 24, True), ("PSL(2,7)", 1, 0.05, 12, True), ("PSL(2,7)", 0, 0.03, 12, False),
    ("PSL(2,11)", 0, 0.03, 5, True), ("PSL(2,11)", 1, 0.02, 4, False)])
def test_decode_16bit_bit_exact(codes, L, precision, name, side, p, shots, use_lead):
    inst, code, oc = codes[name]
    e, syn = _syn(oc, side, shots, p, 11)
    corr, st, it, post = _decode(L, code, side, syn, p, precision, use_lead=use_lead)
    wc, wst, wit, wpost = olead.decode(oc, side, syn, p, use_lead=use_lead, precision=precision)
    assert (st == wst).all()
    assert (it == wit).all()
    assert (corr == wc).all()
    assert (post.view(np.uint32) == wpost.view(np.uint32)).all()
    conv = st == L.ST_CONVERGED
    assert (philox.syndromes(oc.sides[side].H, wc)[conv] == syn[conv]).all()


@pytest.mark.parametrize("precision", MODES)
def test_decode_priors_16bit(codes, L, precision):
    inst, code, oc = codes["PSL(2,7)"]
    info = code.info
    side, shots = 0, 8
    prior = workloads.per_qubit_priors(shots, oc.n, 0.03, 0.5, 2)
    e = workloads.errors_from_priors(prior, 2)
    syn = philox.syndromes(oc.sides[side].H, e)
    o = L.opts(side=side, p=0.03, precision=precision)
    ws = torch.zeros(code.priors_workspace_bytes(o, shots) // 4 + 64, dtype=torch.int32, device="cuda")
    lam = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    sd = _dev_words(syn, info.words_m[side])
    pd = torch.from_numpy(prior).cuda()
    code.local_estimate_priors(o, sd, shots, pd, lam, workspace=ws)
    corr = torch.zeros((shots, info.words_n), dtype=torch.int32, device="cuda")
    st = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    it = torch.zeros(shots, dtype=torch.int32, device="cuda")
    post = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    code.decode_priors(o, sd, shots, pd, corr, st, it, post, ws)
    torch.cuda.synchronize()
    wc, wst, wit, wpost = olead.min_sum(oc.sides[side].H, oc.sides[side].m_l, syn, lam.cpu().numpy(), 32,
                                        precision=precision)
    assert (st.cpu().numpy() == wst).all() and (it.cpu().numpy() == wit).all()
    assert (philox.unpack_bits(corr.cpu().numpy().view(np.uint32), info.n) == wc).all()
    assert (post.cpu().numpy().view(np.uint32) == wpost.view(np.uint32)).all()


def test_modes_compile_once_and_reject_unknown(codes, L):
    inst, code, oc = codes["SL(2,3)"]
    e, syn = _syn(oc, 0, 8, 0.04, 1)
    a = _decode(L, code, 0, syn, 0.04, 1)
    b = _decode(L, code, 0, syn, 0.04, 1)           # the cached kernel: same results
    for x, y in zip(a, b):
        assert (np.asarray(x).view(np.uint8) == np.asarray(y).view(np.uint8)).all()
    with pytest.raises(L.LeadError):
        _decode(L, code, 0, syn, 0.04, 3)
