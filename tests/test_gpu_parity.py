"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Bar: integer / bit work (enumerators, ML decisions, errors, syndromes, corrections, status,
iterations, failure flags) bit-exact; binary32 decision-track values (local tables, prior LLRs,
final posteriors) bit-exact with the oracle's binary32 track; prior LLRs within 1e-4 of the
oracle's FP64 values.
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


def _dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _words(bits, words):
    return philox.pack_bits(bits, words).view(np.int32)


def _bits(words_t, nbits):
    return philox.unpack_bits(words_t.cpu().numpy().view(np.uint32), nbits)


@pytest.mark.parametrize("name", ["SL(2,3)", "PSL(2,7)"])
@pytest.mark.parametrize("side", [0, 1])
def test_enumerators_exact(codes, name, side):
    inst, code, oc = codes[name]
    N, N1, ml = code.enumerators(side)
    oN, oN1, oml = olocal.tables(oc.sides[side].RA, oc.sides[side].RB)
    assert (N == oN).all()
    assert (N1 == oN1).all()
    assert (ml.astype(np.int64) == oml).all()


@pytest.mark.parametrize("name", ["SL(2,3)", "PSL(2,7)"])
@pytest.mark.parametrize("p", [0.01, 0.05, 0.0266667, 0.3])
def test_local_table_bit_exact(codes, L, name, p):
    inst, code, oc = codes[name]
    for side in (0, 1):
        nl = inst.delta ** 2
        t = torch.zeros((1 << code.info.m_l[side]) * nl, dtype=torch.float32, device="cuda")
        code.local_table(side, p, t)
        torch.cuda.synchronize()
        want = olocal.boosted_table_f32(*olocal.tables(oc.sides[side].RA, oc.sides[side].RB), p)
        got = t.cpu().numpy().reshape(want.shape)
        assert (got.view(np.uint32) == want.view(np.uint32)).all()


@pytest.mark.parametrize("name", ["SL(2,3)", "PSL(2,7)", "PSL(2,11)"])
@pytest.mark.parametrize("noise", [0, 1, 2])
def test_sampler_bit_exact(codes, L, name, noise):
    inst, code, oc = codes[name]
    info = code.info
    shots, offset, seed = 37, 1000003, 0xDEADBEEF12345
    ex = torch.full((shots, info.words_n), -1, dtype=torch.int32, device="cuda")
    ez = torch.full((shots, info.words_n), -1, dtype=torch.int32, device="cuda")
    sz = torch.full((shots, info.words_m[0]), -1, dtype=torch.int32, device="cuda")
    sx = torch.full((shots, info.words_m[1]), -1, dtype=torch.int32, device="cuda")
    p = 0.07
    code.sample(noise, p, shots, seed, offset, err_x=ex, err_z=ez, syn_z=sz, syn_x=sx)
    torch.cuda.synchronize()
    x, z = philox.sample_errors(noise, p, seed, offset + np.arange(shots), oc.n)
    assert (ex.cpu().numpy() == _words(x, info.words_n)).all()
    assert (ez.cpu().numpy() == _words(z, info.words_n)).all()
    assert (sz.cpu().numpy() == _words(philox.syndromes(oc.HZ, x), info.words_m[0])).all()
    assert (sx.cpu().numpy() == _words(philox.syndromes(oc.HX, z), info.words_m[1])).all()


def test_sampler_sampled_rows_at_full_size(codes, L):
    """2^20 shots in one launch; the oracle recomputes 12 sampled rows one by one."""
    inst, code, oc = codes["PSL(2,7)"]
    info = code.info
    shots = 1 << 20
    ex = torch.zeros((shots, info.words_n), dtype=torch.int32, device="cuda")
    sz = torch.zeros((shots, info.words_m[0]), dtype=torch.int32, device="cuda")
    code.sample(0, 0.05, shots, 0, 0, err_x=ex, syn_z=sz)
    torch.cuda.synchronize()
    rows = np.array([0, 1, 777, 4095, 65536, 99991, 500000, 654321, 1000000, shots - 2, shots - 1, 31337])
    x, _ = philox.sample_errors(0, 0.05, 0, rows, oc.n)
    assert (ex[torch.from_numpy(rows).cuda()].cpu().numpy() == _words(x, info.words_n)).all()
    assert (sz[torch.from_numpy(rows).cuda()].cpu().numpy() ==
            _words(philox.syndromes(oc.HZ, x), info.words_m[0])).all()
    # a property at any size: the frequency of flips stays inside its binomial band
    flips = sum(int(torch.bitwise_count(ex[i:i + 65536]).sum()) if hasattr(torch, "bitwise_count") else
                int(np.bitwise_count(ex[i:i + 65536].cpu().numpy().view(np.uint32)).sum())
                for i in range(0, shots, 65536))
    n = shots * oc.n
    assert abs(flips / n - 0.05) < 5 * np.sqrt(0.05 * 0.95 / n)


def _syndromes(oc, side, shots, p, seed=0, offset=0):
    noise = philox.NOISE_X if side == 0 else philox.NOISE_Z
    x, z = philox.sample_errors(noise, p, seed, offset + np.arange(shots), oc.n)
    e = x if side == 0 else z
    return e, philox.syndromes(oc.sides[side].H, e)


@pytest.mark.parametrize("name,side,p,shots", [("SL(2,3)", 0, 0.05, 45), ("SL(2,3)", 1, 0.08, 33),
                                               ("PSL(2,7)", 0, 0.03, 21), ("PSL(2,7)", 1, 0.05, 19),
                                               ("PSL(2,11)", 0, 0.03, 7)])
def test_local_estimate_llr(codes, L, name, side, p, shots):
    inst, code, oc = codes[name]
    info = code.info
    e, syn = _syndromes(oc, side, shots, p, seed=5)
    o = L.opts(side=side, p=p, alpha=1.0)
    ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
    llr = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    code.local_estimate(o, _dev(_words(syn, info.words_m[side])), shots, llr, ws)
    torch.cuda.synchronize()
    got = llr.cpu().numpy()
    want32 = olead.prior_f32(oc, side, syn, p)
    _, want64 = olead.prior_f64(oc, side, syn, p)
    assert (got.view(np.uint32) == want32.view(np.uint32)).all()
    assert np.abs(got.astype(np.float64) - want64).max() <= 1e-4


def _decode(L, code, oc, side, syn, p, alpha=1.0, max_iter=32, use_lead=True):
    info = code.info
    shots = syn.shape[0]
    o = L.opts(side=side, p=p, alpha=alpha, max_iter=max_iter, use_lead=use_lead)
    ws = torch.zeros(max(code.workspace_bytes(o), 256) // 4 + 64, dtype=torch.int32, device="cuda")
    corr = torch.full((shots, info.words_n), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    it = torch.full((shots,), -1, dtype=torch.int32, device="cuda")
    llr = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    code.decode(o, _dev(_words(syn, info.words_m[side])), shots, corr, st, it, llr, ws)
    torch.cuda.synchronize()
    return corr, st.cpu().numpy(), it.cpu().numpy(), llr.cpu().numpy()


@pytest.mark.parametrize("name,side,p,shots,use_lead", [
    ("SL(2,3)", 0, 0.04, 67, True), ("SL(2,3)", 1, 0.08, 41, True), ("SL(2,3)", 0, 0.06, 50, False),
    ("PSL(2,7)", 0, 0.01, 40, True), ("PSL(2,7)", 0, 0.02, 40, True), ("PSL(2,7)", 1, 0.03, 24, True),
    ("PSL(2,7)", 0, 0.05, 12, True), ("PSL(2,7)", 0, 0.02, 20, False),
    # |G| = 660: the decoder runs one shot per thread-block cluster
    ("PSL(2,11)", 0, 0.03, 9, True), ("PSL(2,11)", 1, 0.02, 7, True), ("PSL(2,11)", 0, 0.02, 5, False)])
def test_decode_bit_exact(codes, L, name, side, p, shots, use_lead):
    inst, code, oc = codes[name]
    info = code.info
    e, syn = _syndromes(oc, side, shots, p, seed=11)
    corr, st, it, post = _decode(L, code, oc, side, syn, p, use_lead=use_lead)
    wc, wst, wit, wpost = olead.decode(oc, side, syn, p, use_lead=use_lead)
    assert (st == wst).all()
    assert (it == wit).all()
    assert (_bits(corr, oc.n) == wc).all()
    assert (corr.cpu().numpy() == _words(wc, info.words_n)).all()      # padding bits are zero
    assert (post.view(np.uint32) == wpost.view(np.uint32)).all()
    # the paper's output contract: a converged correction satisfies H e = s
    conv = st == L.ST_CONVERGED
    assert (philox.syndromes(oc.sides[side].H, wc)[conv] == syn[conv]).all()


@pytest.mark.parametrize("p", [0.02, 0.05, 0.08])
def test_sl3_workload_every_shot(codes, L, p):
    """The SL(2,3) workload in full: X noise at p = 0.02, 0.05, 0.08 with 10^4 shots each,
    binary32 LEAD. Every shot's correction, status, iteration count, posterior and check flag
    equals the oracle's."""
    inst, code, oc = codes["SL(2,3)"]
    info = code.info
    shots = 10_000
    e, syn = _syndromes(oc, 0, shots, p, seed=0)
    corr, st, it, post = _decode(L, code, oc, 0, syn, p)
    wc, wst, wit, wpost = olead.decode(oc, 0, syn, p)
    assert (st == wst).all() and (it == wit).all()
    assert (_bits(corr, oc.n) == wc).all()
    assert (post.view(np.uint32) == wpost.view(np.uint32)).all()
    fail = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    code.check(0, _dev(_words(e, info.words_n)), corr, shots, fail)
    assert (fail.cpu().numpy() == olead.check(oc, 0, e, wc)).all()


def test_decode_alpha_and_max_iter_edges(codes, L):
    inst, code, oc = codes["PSL(2,7)"]
    e, syn = _syndromes(oc, 0, 9, 0.02, seed=3)
    for alpha, mi in ((0.01, 32), (1.0, 0), (0.5, 3)):
        corr, st, it, post = _decode(L, code, oc, 0, syn, 0.02, alpha=alpha, max_iter=mi)
        wc, wst, wit, wpost = olead.decode(oc, 0, syn, 0.02, alpha=alpha, max_iter=mi)
        assert (st == wst).all() and (it == wit).all() and (_bits(corr, oc.n) == wc).all()
        assert (post.view(np.uint32) == wpost.view(np.uint32)).all()


def test_zero_syndrome_and_empty_batch(codes, L):
    inst, code, oc = codes["PSL(2,7)"]
    syn = np.zeros((5, oc.HZ.shape[0]), dtype=np.uint8)
    corr, st, it, _ = _decode(L, code, oc, 0, syn, 0.05)
    assert not corr.cpu().numpy().any() and (st == L.ST_CONVERGED).all() and (it == 0).all()
    o = L.opts(side=0, p=0.05)
    ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
    empty = torch.zeros((0, code.info.words_m[0]), dtype=torch.int32, device="cuda")
    code.decode(o, empty, 0, empty, torch.zeros(0, dtype=torch.uint8, device="cuda"), workspace=ws)


def test_invalid_options_rejected(codes, L):
    inst, code, oc = codes["PSL(2,7)"]
    for kw in (dict(p=0.6), dict(alpha=0.0), dict(max_iter=65)):
        o = L.opts(side=0, **{**dict(p=0.05), **kw})
        with pytest.raises(L.LeadError) as e:
            code.decode(o, torch.zeros((1, 48), dtype=torch.int32, device="cuda"), 1,
                        torch.zeros((1, 96), dtype=torch.int32, device="cuda"),
                        torch.zeros(1, dtype=torch.uint8, device="cuda"),
                        workspace=torch.zeros(30000, dtype=torch.int32, device="cuda"))
        assert e.value.rc == -1


@pytest.mark.parametrize("name", ["SL(2,3)", "PSL(2,7)", "PSL(2,11)"])
def test_check_flags_exact(codes, L, name):
    inst, code, oc = codes[name]
    info = code.info
    shots = 60 if name != "PSL(2,11)" else 6
    for side in (0, 1):
        e, syn = _syndromes(oc, side, shots, 0.05, seed=17)
        wc, wst, wit, _ = olead.decode(oc, side, syn, 0.05)
        # also plant known residuals: a stabilizer (no failure) and a logical (failure)
        from oracle import gf2
        other = oc.sides[1 - side].H
        ker = gf2.kernel_basis(oc.sides[side].H)
        rs = gf2.RowSpace(other)
        logical = next(v for v in ker if not rs.contains(v))
        wc = wc.copy()
        wc[0] = e[0] ^ other[0]
        wc[1] = e[1] ^ logical
        fail = torch.zeros(shots, dtype=torch.uint8, device="cuda")
        code.check(side, _dev(_words(e, info.words_n)), _dev(_words(wc, info.words_n)), shots, fail)
        torch.cuda.synchronize()
        want = olead.check(oc, side, e, wc)
        assert (fail.cpu().numpy() == want).all()
        assert want[0] == 0 and want[1] == 2


def test_pipeline_counts_match_oracle(codes, L):
    """End-to-end through the batched driver (several chunks, ragged tail) on SL(2,3)."""
    from paper_2605_17796_gb300.pipeline import Pipeline
    inst, code, oc = codes["SL(2,3)"]
    pipe = Pipeline(code, chunk=128)
    shots, p = 300, 0.05
    r = pipe.run(philox.NOISE_DEPOL, p, shots, seed=9, offset=0)
    x, z = philox.sample_errors(philox.NOISE_DEPOL, p, 9, np.arange(shots), oc.n)
    fails = np.zeros(shots, dtype=bool)
    its = 0
    for side, e in ((0, x), (1, z)):
        syn = philox.syndromes(oc.sides[side].H, e)
        wc, wst, wit, _ = olead.decode(oc, side, syn, 2 * p / 3)
        fails |= olead.check(oc, side, e, wc) != 0
        its += int(wit.sum())
    assert r.failures == int(fails.sum())
    assert r.iters_sum == its


@pytest.mark.parametrize("GA,expect", [
    # local codes whose boosted posteriors take more distinct values than the shared pair
    # table holds (79 classes) or than a class byte holds (1 581): both take the direct merge
    ([[1, 1, 0, 1, 1, 0], [0, 1, 1, 0, 1, 1], [1, 0, 0, 1, 0, 1]], 79),
    ([[1, 1, 0, 1, 1, 1], [1, 1, 1, 0, 1, 0], [1, 1, 1, 1, 0, 0]], 1581)])
@pytest.mark.parametrize("precision", [0, 1])
def test_local_estimate_many_classes(L, GA, expect, precision):
    import dataclasses
    inst = dataclasses.replace(workloads.standard("PSL(2,7)", 0), GA=np.array(GA, dtype=np.uint8))
    oc = tanner.from_instance(inst)
    N, N1, ml = olocal.tables(oc.sides[0].RA, oc.sides[0].RB)
    assert len(np.unique(olocal.boosted_table_f32(N, N1, ml, 0.05).view(np.uint32))) == expect
    code = L.Code.from_instance(inst).prepare(0)
    info = code.info
    shots, p = 70, 0.05
    e, syn = _syndromes(oc, 0, shots, p, seed=4)
    o = L.opts(side=0, p=p, precision=precision)
    ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
    llr = torch.zeros((shots, info.n), dtype=torch.float32 if precision == 0 else torch.int16, device="cuda")
    code.local_estimate(o, _dev(_words(syn, info.words_m[0])), shots, llr, ws)
    torch.cuda.synchronize()
    want = olead.round_storage(olead.prior_f32(oc, 0, syn, p), precision)
    got = llr.cpu().numpy()
    if precision == 1:
        got = (got.view(np.uint16).astype(np.uint32) << 16).view(np.float32)
    assert (got.view(np.uint32) == want.view(np.uint32)).all()


@pytest.mark.parametrize("precision", [0, 2])
def test_local_estimate_unaligned_output(codes, L, precision):
    """An output buffer that starts one element past an allocation boundary gets the same
    values as an aligned one."""
    inst, code, oc = codes["PSL(2,7)"]
    info = code.info
    shots, p = 37, 0.04
    e, syn = _syndromes(oc, 0, shots, p, seed=8)
    o = L.opts(side=0, p=p, precision=precision)
    ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
    dt = torch.float32 if precision == 0 else torch.int16
    sd = _dev(_words(syn, info.words_m[0]))
    a = torch.zeros((shots, info.n), dtype=dt, device="cuda")
    code.local_estimate(o, sd, shots, a, ws)
    big = torch.zeros(shots * info.n + 1, dtype=dt, device="cuda")
    b = big[1:].view(shots, info.n)
    code.local_estimate(o, sd, shots, b, ws)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    want = olead.round_storage(olead.prior_f32(oc, 0, syn, p), precision)
    got = a.cpu().numpy()
    if precision == 2:
        got = got.view(np.float16).astype(np.float32)
    assert (got.view(np.uint32) == want.view(np.uint32)).all()
