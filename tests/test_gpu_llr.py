"""The prior LLR lambda(p) = ln((1-p)/p) of the CUDA path (lead_prior_llr, the conversion every
decode call applies) against the oracle's plain definition (the binary32 rounding of the exact
value), on every binary32 input of the clamp range [2^-23, 1/2] and on sampled inputs above 1/2.

Bar: equal bit for bit except on a stated set of inputs, each at most 1 ulp away. The GPU
evaluates in binary32 pairs (about 2^-45 relative before the final rounding); an exhaustive run
of the same arithmetic found 3 of the 184 549 377 inputs within that distance of a rounding
boundary, and those are the only ones allowed to differ.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LO, HI = 0x34000000, 0x3F000000          # bit patterns of 2^-23 and 1/2
CHUNK = 1 << 24
# inputs whose binary32-pair value lies within its error of a rounding boundary (1 ulp off)
KNOWN_OFF = {0x3489CC36, 0x35C418A7, 0x3B4E9C2C}


def _oracle_chunk(start, stop):
    import numpy as np
    from oracle import local
    u = np.arange(start, stop, dtype=np.uint32)
    return local.llr_f32(u.view(np.float32)).view(np.uint32)


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2605_17796_gb300 import lead
    return lead


def _gpu(L, start, stop):
    u = torch.arange(start, stop, dtype=torch.int64, device="cuda").to(torch.int32)
    p = u.view(torch.float32)
    out = torch.empty_like(p)
    L.prior_llr(p, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def test_prior_llr_every_binary32_input(L):
    ranges = [(s, min(s + CHUNK, HI + 1)) for s in range(LO, HI + 1, CHUNK)]
    off = []
    with cf.ProcessPoolExecutor(max_workers=min(16, len(ranges)), mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_oracle_chunk, a, b) for a, b in ranges]
        for (a, b), f in zip(ranges, futs):
            got = _gpu(L, a, b)
            want = f.result()
            bad = np.nonzero(got != want)[0]
            for k in bad:
                assert abs(int(got[k]) - int(want[k])) == 1, hex(a + int(k))
            off.extend(int(a + k) for k in bad)
    assert set(off) <= KNOWN_OFF, [hex(x) for x in off]
    assert len(off) <= 3


def test_prior_llr_above_half_and_edges(L):
    # p in (1/2, 1 - 2^-23]: lambda(p) = -lambda(1 - p) with 1 - p exact; sampled every 7th input
    u = np.arange(0x3F000001, 0x3F7FFFFF, 7, dtype=np.uint32)
    p = u.view(np.float32)
    pt = torch.from_numpy(p.copy()).cuda()
    out = torch.empty_like(pt)
    L.prior_llr(pt, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    from oracle import local
    assert (got.view(np.uint32) == local.llr_f32(p).view(np.uint32)).all()
    q = (np.float32(1) - p).astype(np.float32)
    assert (got == -local.llr_f32(q)).all()
    # clamp, the midpoint, and an empty call
    edge = torch.tensor([0.0, -1.0, 1.0, 2.0, 0.5, 2.0 ** -23, 1 - 2.0 ** -23], dtype=torch.float32, device="cuda")
    eo = torch.empty_like(edge)
    L.prior_llr(edge, eo)
    torch.cuda.synchronize()
    want = local.llr_f32(edge.cpu().numpy())
    assert (eo.cpu().numpy().view(np.uint32) == want.view(np.uint32)).all()
    assert eo[4].item() == 0.0
    L.prior_llr(torch.empty(0, device="cuda"), torch.empty(0, device="cuda"))
