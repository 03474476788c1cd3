"""Per-qubit priors (lead_local_estimate_priors / lead_decode_priors) against the oracle.

Bar:
* least-cost local decisions (integer costs W_j = rint(2^20 lambda(p_j)), exact sums): bit-exact;
* boosted local posteriors: relative error <= 1e-4 against the oracle's FP64 posterior of the
  exact priors. The kernel takes lambda(p) rounded to binary32 (relative error 2^-24), sums at
  most 6 of them per row pattern and 6 row log-sums per coset member in binary32, and evaluates
  the log-sum-exps in binary32: every exponent is within about 1e-5 of its exact value, so every
  term and every ratio q = num / Z stays within about 2e-5;
* merged prior LLRs: bit-exact with the oracle's binary32 merge applied to the kernel's own
  posteriors;
* the whole decode from the raw priors and syndromes: the oracle runs its own FP64 local
  posteriors, the binary32 merge and min-sum. A posterior that differs from the kernel's in its
  last bits can move a merged LLR by an ulp and change a min-sum trajectory (most visibly in
  shots that do not converge, whose last decision wanders), so two counts are held under stated
  bounds: shots whose decoder-failure verdict differs, and shots converged on both sides with
  different corrections; the count of shots with any difference is printed. With use_lead = 0
  (the prior LLR alone) the decode is bit-exact.
"""
import numpy as np
import pytest

import workloads
from oracle import lead as olead
from oracle import local as olocal
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


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _inputs(oc, side, shots, p, seed):
    prior = workloads.per_qubit_priors(shots, oc.n, p, 0.5, seed)
    e = workloads.errors_from_priors(prior, seed)
    return prior, e, philox.syndromes(oc.sides[side].H, e)


def _estimate(L, code, side, syn, prior, alpha=1.0, with_q=True):
    info = code.info
    shots = syn.shape[0]
    o = L.opts(side=side, p=0.05, alpha=alpha)
    llr = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    q = torch.zeros((shots, info.order, info.delta ** 2), dtype=torch.float32, device="cuda") if with_q else None
    ml = torch.zeros((shots, info.order), dtype=torch.int64, device="cuda")
    ws = torch.zeros(code.priors_workspace_bytes(o, shots) // 4 + 64, dtype=torch.int32, device="cuda")
    code.local_estimate_priors(o, _dev(philox.pack_bits(syn, info.words_m[side]).view(np.int32)), shots,
                               _dev(prior), llr, q=q, ml=ml, workspace=ws)
    torch.cuda.synchronize()
    return (llr.cpu().numpy(), q.cpu().numpy() if with_q else None,
            ml.cpu().numpy().view(np.uint64).astype(np.int64))


@pytest.mark.parametrize("name,side,p,shots", [("SL(2,3)", 0, 0.05, 9), ("SL(2,3)", 1, 0.1, 7),
                                               ("PSL(2,7)", 0, 0.03, 2), ("PSL(2,7)", 1, 0.06, 2)])
def test_local_priors_parity(codes, L, name, side, p, shots):
    inst, code, oc = codes[name]
    prior, e, syn = _inputs(oc, side, shots, p, seed=7)
    llr, q, ml = _estimate(L, code, side, syn, prior)
    want_q, want_ml = olead.local_priors(oc, side, syn, prior)
    assert (ml == want_ml).all()
    rel = np.abs(q - want_q) / np.maximum(want_q, 1e-30)
    print(f"{name} side {side}: max relative error of q against FP64 {rel.max():.2e}")
    assert np.all(np.abs(q - want_q) <= 1e-4 * want_q + 1e-30)
    # every least-cost decision satisfies its local syndrome
    Hl = np.kron(oc.sides[side].RB, oc.sides[side].RA).astype(np.int64)
    sv = olead.local_syndromes(oc.sides[side], syn)
    bits = (ml[..., None] >> np.arange(inst.delta ** 2)) & 1
    s_of = ((bits @ Hl.T) & 1) @ (1 << np.arange(Hl.shape[0]))
    assert (s_of == sv).all()
    got_merge = olead.merge_priors_f32(oc, side, q.astype(np.float64))
    assert (llr.view(np.uint32) == got_merge.view(np.uint32)).all()


@pytest.mark.parametrize("name", ["SL(2,3)", "PSL(2,7)"])
def test_uniform_priors_reduce_to_table_path(codes, L, name):
    inst, code, oc = codes[name]
    p = 0.04
    for side in (0, 1):
        e = philox.sample_errors(side, p, 3, np.arange(4), oc.n)[side]
        syn = philox.syndromes(oc.sides[side].H, e)
        prior = np.full((4, oc.n), p, dtype=np.float32)
        llr, q, ml = _estimate(L, code, side, syn, prior)
        N, N1, oml = olocal.tables(oc.sides[side].RA, oc.sides[side].RB)
        sv = olead.local_syndromes(oc.sides[side], syn)
        assert (ml == oml[sv]).all()                                  # least cost = least weight
        table = olocal.boosted_table_f32(N, N1, oml, p).astype(np.float64)
        want = table[sv]
        assert np.all(np.abs(q - want) <= 1e-4 * want + 1e-30)


def _decode_priors(L, code, side, syn, prior, use_lead=True, alpha=1.0, max_iter=32):
    info = code.info
    shots = syn.shape[0]
    o = L.opts(side=side, p=0.05, alpha=alpha, max_iter=max_iter, use_lead=use_lead)
    ws = torch.zeros(code.priors_workspace_bytes(o, shots) // 4 + 64, dtype=torch.int32, device="cuda")
    corr = torch.full((shots, info.words_n), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    it = torch.full((shots,), -1, dtype=torch.int32, device="cuda")
    post = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    code.decode_priors(o, _dev(philox.pack_bits(syn, info.words_m[side]).view(np.int32)), shots, _dev(prior),
                       corr, st, it, post, ws)
    torch.cuda.synchronize()
    return (philox.unpack_bits(corr.cpu().numpy().view(np.uint32), code.info.n), st.cpu().numpy(),
            it.cpu().numpy(), post.cpu().numpy())


# fractions of the decoded shots allowed a different failure verdict, and a different correction
# among the shots converged on both sides, against the oracle run from raw inputs
VERDICT_BOUND = 0.05
CONVERGED_BOUND = 0.05


@pytest.mark.parametrize("name,side,p,shots,use_lead", [
    ("SL(2,3)", 0, 0.05, 200, True), ("SL(2,3)", 1, 0.08, 60, False),
    ("PSL(2,7)", 0, 0.02, 40, True), ("PSL(2,7)", 1, 0.03, 40, True), ("PSL(2,7)", 0, 0.03, 20, False),
    ("PSL(2,11)", 0, 0.02, 3, True), ("PSL(2,11)", 1, 0.02, 3, False)])
def test_decode_priors_from_raw_inputs(codes, L, name, side, p, shots, use_lead):
    inst, code, oc = codes[name]
    prior, e, syn = _inputs(oc, side, shots, p, seed=13)
    corr, st, it, post = _decode_priors(L, code, side, syn, prior, use_lead=use_lead)
    if use_lead:
        q, _ = olead.local_priors(oc, side, syn, prior)
        lam = olead.merge_priors_f32(oc, side, q)
    else:
        lam = olocal.llr_f32(prior)
    H = oc.sides[side].H
    wc, wst, wit, wpost = olead.min_sum(H, oc.sides[side].m_l, syn, lam, 32)
    conv = st == L.ST_CONVERGED
    assert (philox.syndromes(H, corr)[conv] == syn[conv]).all()
    if not use_lead:
        assert (st == wst).all() and (it == wit).all() and (corr == wc).all()
        assert (post.view(np.uint32) == wpost.view(np.uint32)).all()
        return
    bad = (st != wst) | (it != wit) | (corr != wc).any(axis=1)
    verdict = int((st != wst).sum())
    both = (st == L.ST_CONVERGED) & (wst == L.ST_CONVERGED)
    conv_diff = int(((corr != wc).any(axis=1) & both).sum())
    print(f"{name} side {side} p={p}: {int(bad.sum())}/{shots} shots differ from the oracle run from raw "
          f"inputs; failure verdicts differ on {verdict}; converged on both {int(both.sum())}, of them with "
          f"different corrections {conv_diff}")
    assert verdict <= max(1, int(VERDICT_BOUND * shots))
    assert conv_diff <= max(1, int(CONVERGED_BOUND * shots))


def test_decode_priors_bit_exact_on_its_own_llrs(codes, L):
    """Phase 3 alone: min-sum from the kernel's own merged LLRs equals the oracle's, bit for bit."""
    inst, code, oc = codes["PSL(2,7)"]
    prior, e, syn = _inputs(oc, 0, 12, 0.02, seed=13)
    corr, st, it, post = _decode_priors(L, code, 0, syn, prior)
    lam, _, _ = _estimate(L, code, 0, syn, prior, with_q=False)
    wc, wst, wit, wpost = olead.min_sum(oc.sides[0].H, oc.sides[0].m_l, syn, lam, 32)
    assert (st == wst).all() and (it == wit).all() and (corr == wc).all()
    assert (post.view(np.uint32) == wpost.view(np.uint32)).all()


def test_passes_split_large_batches(codes, L):
    """A batch larger than one pass of the workspace: every row equals the same row decoded
    alone (rows at and around the pass boundary included), and sampled rows match the oracle."""
    inst, code, oc = codes["PSL(2,7)"]
    side, p = 0, 0.02
    per_shot = oc.n * 4 + inst.delta ** 2 * len(oc.sides[0].views) * 4
    boundary = (256 << 20) // per_shot
    shots = boundary + 40
    prior, e, syn = _inputs(oc, side, shots, p, seed=17)
    llr, _, ml = _estimate(L, code, side, syn, prior, with_q=False)
    corr, st, it, post = _decode_priors(L, code, side, syn, prior)
    rows = np.array([0, 1, boundary - 1, boundary, boundary + 1, shots - 1])
    llr_r, q_r, ml_r = _estimate(L, code, side, syn[rows], prior[rows])
    assert (llr[rows].view(np.uint32) == llr_r.view(np.uint32)).all()
    assert (ml[rows] == ml_r).all()
    c_r, st_r, it_r, post_r = _decode_priors(L, code, side, syn[rows], prior[rows])
    assert (corr[rows] == c_r).all() and (st[rows] == st_r).all() and (it[rows] == it_r).all()
    assert (post[rows].view(np.uint32) == post_r.view(np.uint32)).all()
    want_q, want_ml = olead.local_priors(oc, side, syn[rows[[2, 3]]], prior[rows[[2, 3]]])
    assert (ml_r[[2, 3]] == want_ml).all()
    assert np.all(np.abs(q_r[[2, 3]] - want_q) <= 1e-4 * want_q + 1e-30)


def test_priors_edges(codes, L):
    inst, code, oc = codes["PSL(2,7)"]
    info = code.info
    o = L.opts(side=0, p=0.05)
    ws = torch.zeros(1024, dtype=torch.int32, device="cuda")
    empty = torch.zeros((0, info.words_m[0]), dtype=torch.int32, device="cuda")
    # empty batch: nothing read or written
    code.decode_priors(o, empty, 0, torch.zeros((0, info.n), device="cuda"), empty,
                       torch.zeros(0, dtype=torch.uint8, device="cuda"), workspace=ws)
    # zero syndrome: the least-cost decision is zero, the decoder converges at iteration 0
    syn = np.zeros((3, oc.sides[0].H.shape[0]), dtype=np.uint8)
    prior = workloads.per_qubit_priors(3, oc.n, 0.05, 0.9, 1)
    corr, st, it, _ = _decode_priors(L, code, 0, syn, prior)
    assert not corr.any() and (st == L.ST_CONVERGED).all() and (it == 0).all()
    _, _, ml = _estimate(L, code, 0, syn, prior, with_q=False)
    assert not ml.any()
    # a too small workspace and a non-fp32 precision are rejected
    small = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(L.LeadError):
        code.decode_priors(o, _dev(philox.pack_bits(syn, info.words_m[0]).view(np.int32)), 3, _dev(prior),
                           torch.zeros((3, info.words_n), dtype=torch.int32, device="cuda"),
                           torch.zeros(3, dtype=torch.uint8, device="cuda"), workspace=small)
