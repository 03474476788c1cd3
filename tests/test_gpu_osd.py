"""OSD-CS post-processing (lead_osd) against the oracle (oracle/osd.py).

The oracle gets the same inputs the kernel got: the syndromes, the device min-sum posteriors
and the device prior LLRs. Corrections and status are compared bit for bit; converged shots must
be left untouched, and every OSD output must satisfy its syndrome.
"""
import numpy as np
import pytest

import workloads
from oracle import osd as oosd
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


def _run(L, code, oc, side, p, shots, order, use_lead=True, seed=3, slots_ws=None):
    info = code.info
    x, z = philox.sample_errors(side, p, seed, np.arange(shots), oc.n)
    e = x if side == 0 else z
    syn = philox.syndromes(oc.sides[side].H, e)
    sd = torch.from_numpy(philox.pack_bits(syn, info.words_m[side]).view(np.int32)).cuda()
    o = L.opts(side=side, p=p, use_lead=use_lead)
    ws = torch.zeros(max(code.workspace_bytes(o), 256) // 4 + 64, dtype=torch.int32, device="cuda")
    corr = torch.zeros((shots, info.words_n), dtype=torch.int32, device="cuda")
    st = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    post = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    code.decode(o, sd, shots, corr, st, None, post, ws)
    prior = None
    if use_lead:
        prior = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
        code.local_estimate(o, sd, shots, prior, ws)
    torch.cuda.synchronize()
    corr0, st0 = corr.clone(), st.clone()
    nb = code.osd_workspace_bytes(o, shots) if slots_ws is None else slots_ws
    ows = torch.zeros(nb // 4 + 64, dtype=torch.int32, device="cuda")
    code.osd(o, order, sd, shots, post, st, corr, prior=prior, workspace=ows)
    torch.cuda.synchronize()
    post_h = post.cpu().numpy()
    prior_h = (prior.cpu().numpy() if prior is not None else
               np.broadcast_to(np.float32(np.log((1 - np.float32(p)) / np.float32(p))), post_h.shape))
    return syn, e, corr0, st0, corr, st, post_h, prior_h


def _channel_prior(p, shape):
    from oracle import local
    return np.broadcast_to(local.llr_f32(np.array([p], dtype=np.float32)), shape).copy()


@pytest.mark.parametrize("name,side,p,shots,order", [("SL(2,3)", 0, 0.08, 60, 3), ("SL(2,3)", 1, 0.06, 50, 0),
                                                     ("SL(2,3)", 0, 0.05, 40, 6), ("PSL(2,7)", 0, 0.03, 5, 3)])
def test_osd_bit_exact(codes, L, name, side, p, shots, order):
    inst, code, oc = codes[name]
    syn, e, corr0, st0, corr, st, post, prior = _run(L, code, oc, side, p, shots, order)
    H = oc.sides[side].H
    conv = (st0.cpu().numpy() & L.ST_CONVERGED) != 0
    assert (~conv).any()
    want, idx = oosd.osd_batch(H, syn, post, prior, order, only=~conv)
    got = philox.unpack_bits(corr.cpu().numpy().view(np.uint32), oc.n)
    before = philox.unpack_bits(corr0.cpu().numpy().view(np.uint32), oc.n)
    assert (got[conv] == before[conv]).all()
    assert (got[~conv] == want[~conv]).all()
    stn = st.cpu().numpy()
    assert (stn[conv] == st0.cpu().numpy()[conv]).all()
    assert ((stn[~conv] & L.ST_OSD) != 0).all()
    assert (philox.syndromes(H, got) == syn).all()
    # padding bits of the correction rows stay zero
    assert (corr.cpu().numpy() == philox.pack_bits(got, code.info.words_n).view(np.int32)).all()


def test_osd_on_the_baseline_uses_the_channel_prior(codes, L):
    inst, code, oc = codes["SL(2,3)"]
    syn, e, corr0, st0, corr, st, post, _ = _run(L, code, oc, 0, 0.07, 50, 3, use_lead=False)
    conv = (st0.cpu().numpy() & L.ST_CONVERGED) != 0
    want, _ = oosd.osd_batch(oc.sides[0].H, syn, post, _channel_prior(0.07, post.shape), 3, only=~conv)
    got = philox.unpack_bits(corr.cpu().numpy().view(np.uint32), oc.n)
    assert (got[~conv] == want[~conv]).all()


def test_one_slot_gives_the_same_result(codes, L):
    inst, code, oc = codes["SL(2,3)"]
    info = code.info
    slot = -(-(oc.sides[0].H.shape[0] * ((oc.n + 63) // 64) * 8) // 256) * 256
    a = _run(L, code, oc, 0, 0.08, 40, 3, seed=9)
    b = _run(L, code, oc, 0, 0.08, 40, 3, seed=9, slots_ws=slot)
    assert torch.equal(a[4], b[4]) and torch.equal(a[5], b[5])


def test_pipeline_with_osd_leaves_no_decoder_failures(codes, L):
    """With OSD after min-sum every correction satisfies its syndrome, so every remaining failure
    is a logical error; without OSD the same shots show decoder failures."""
    from paper_2605_17796_gb300.pipeline import Pipeline
    inst, code, oc = codes["PSL(2,7)"]
    pipe = Pipeline(code, 4096, 0)
    plain = pipe.run(L.NOISE_X, 0.03, 3000, seed=2)
    with_osd = pipe.run(L.NOISE_X, 0.03, 3000, seed=2, osd_order=3)
    assert plain.failures > plain.logical
    assert with_osd.failures == with_osd.logical
    assert with_osd.failures < plain.failures


def test_osd_large_code(codes, L):
    """PSL(2,11) (n = 11 880, m = 5 940): the sort and per-column arrays no longer fit in shared
    memory and live in each slot's global scratch, and every row spans 186 words. Two
    unconverged shots against the oracle (about 30 s of CPU each), all OSD outputs satisfy their
    syndromes, and a one-slot workspace gives the same result."""
    inst, code, oc = codes["PSL(2,11)"]
    H = oc.sides[0].H
    syn, e, corr0, st0, corr, st, post, prior = _run(L, code, oc, 0, 0.04, 6, 3, seed=5)
    conv = (st0.cpu().numpy() & L.ST_CONVERGED) != 0
    redo = np.nonzero(~conv)[0]
    assert redo.size >= 2
    only = np.zeros(len(conv), dtype=bool)
    only[redo[:2]] = True
    want, _ = oosd.osd_batch(H, syn, post, prior, 3, only=only)
    got = philox.unpack_bits(corr.cpu().numpy().view(np.uint32), oc.n)
    assert (got[only] == want[only]).all()
    before = philox.unpack_bits(corr0.cpu().numpy().view(np.uint32), oc.n)
    assert (got[conv] == before[conv]).all()
    assert ((st.cpu().numpy()[~conv] & L.ST_OSD) != 0).all()
    assert (philox.syndromes(H, got) == syn).all()
    o = L.opts(side=0, p=0.04)
    one = code.osd_workspace_bytes(o, 1)
    assert code.osd_workspace_bytes(o, 6) == 6 * one
    b = _run(L, code, oc, 0, 0.04, 6, 3, seed=5, slots_ws=one)
    assert torch.equal(corr, b[4]) and torch.equal(st, b[5])
