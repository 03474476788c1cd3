"""The non-allocating decode entry point (lead_decode_noalloc).

Callers that cannot allocate device memory -- a real-time decode loop with a deadline too short
for cudaMalloc, or a host application whose pool allocator owns all device memory -- use this
entry point; it keeps the per-call tables (the local posterior table and its class tables) in a
fixed array inside the library instead of a caller workspace. This file runs last, so a run that
stops at the first failure has run every other test.

* two calls in a row through the C ABI (two noise levels, so the second call must overwrite the
  first call's tables) give lead_decode's outputs bit for bit, and the device's free memory is
  the same before and after them;
* a local code whose tables exceed LEAD_NOALLOC_TABLE_BYTES is rejected with LEAD_EINVAL;
* an empty batch returns at once, as lead_decode does.
"""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2605_17796_gb300 import lead
    return lead


def _outs(L, code, o, sz, shots, noalloc, ws=None):
    info = code.info
    corr = torch.full((shots, info.words_n), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    it = torch.full((shots,), -1, dtype=torch.int32, device="cuda")
    llr = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    if noalloc:
        code.decode_noalloc(o, sz, shots, corr, st, it, llr)
    else:
        code.decode(o, sz, shots, corr, st, it, llr, workspace=ws)
    torch.cuda.synchronize()
    return corr.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy(), llr.cpu().numpy()


def test_noalloc_matches_decode_on_two_calls(L):
    import workloads
    inst = workloads.standard("PSL(2,7)", 0)
    code = L.Code.from_instance(inst).prepare(0)
    info = code.info
    shots = 300
    ex = torch.zeros((shots, info.words_n), dtype=torch.int32, device="cuda")
    sz = torch.zeros((2, shots, info.words_m[0]), dtype=torch.int32, device="cuda")
    ps = (0.05, 0.02)
    refs = []
    for call, p in enumerate(ps):
        code.sample(L.NOISE_X, p, shots, 123 + call, 0, err_x=ex, syn_z=sz[call])
        o = L.opts(side=0, p=p)
        ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
        refs.append(_outs(L, code, o, sz[call], shots, False, ws))
    # the two non-allocating calls back to back, with every output buffer made beforehand
    bufs = [(torch.full((shots, info.words_n), -1, dtype=torch.int32, device="cuda"),
             torch.zeros(shots, dtype=torch.uint8, device="cuda"),
             torch.full((shots,), -1, dtype=torch.int32, device="cuda"),
             torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")) for _ in ps]
    torch.cuda.synchronize()
    code.decode_noalloc(L.opts(side=0, p=ps[0]), sz[0], 1, *[b[:1] for b in bufs[0]])   # per-device set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for call, p in enumerate(ps):
        code.decode_noalloc(L.opts(side=0, p=p), sz[call], shots, *bufs[call])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, "the non-allocating calls changed the device's free memory"
    for (c0, s0, i0, l0), b in zip(refs, bufs):
        c1, s1, i1, l1 = (t.cpu().numpy() for t in b)
        assert (c0 == c1).all() and (s0 == s1).all() and (i0 == i1).all()
        assert (l0.view(np.uint32) == l1.view(np.uint32)).all()
        assert (s1 == L.ST_CONVERGED).any()


def test_noalloc_rejects_oversize_tables_and_accepts_empty_batches(L):
    import workloads
    base = workloads.standard("PSL(2,7)", 0)
    # C_B of dimension 4 instead of C_A^perp: side 0 has k_A k_B = 12 local checks, so its
    # tables (2^12 x 36 floats and their classes) exceed the fixed array
    GB = np.array([[1, 0, 0, 0, 1, 1], [0, 1, 0, 0, 1, 0], [0, 0, 1, 0, 0, 1], [0, 0, 0, 1, 1, 1]], dtype=np.uint8)
    code = L.Code.from_instance(dataclasses.replace(base, GB=GB)).prepare(0)
    info = code.info
    assert info.m_l[0] == 12
    o = L.opts(side=0, p=0.05)
    assert code.workspace_bytes(o) > L.NOALLOC_TABLE_BYTES
    sz = torch.zeros((4, info.words_m[0]), dtype=torch.int32, device="cuda")
    bufs = (torch.zeros((4, info.words_n), dtype=torch.int32, device="cuda"),
            torch.zeros(4, dtype=torch.uint8, device="cuda"))
    with pytest.raises(L.LeadError) as e:
        code.decode_noalloc(o, sz, 4, *bufs)
    assert e.value.rc == -1
    # the channel-prior baseline needs no tables, so the same code decodes
    code.decode_noalloc(L.opts(side=0, p=0.05, use_lead=False), sz, 4, *bufs)
    torch.cuda.synchronize()
    assert (bufs[1].cpu().numpy() == L.ST_CONVERGED).all()      # zero syndromes
    # an empty batch is a no-op, as in lead_decode (the oversize check is not reached)
    empty = torch.zeros((0, info.words_m[0]), dtype=torch.int32, device="cuda")
    code.decode_noalloc(o, empty, 0, torch.zeros((0, info.words_n), dtype=torch.int32, device="cuda"),
                        torch.zeros(0, dtype=torch.uint8, device="cuda"))
