"""The non-allocating decode entry point (lead_decode_noalloc).

Callers that cannot allocate device memory -- a real-time decode loop with a deadline too short
for cudaMalloc, or a host application whose pool allocator owns all device memory -- use this
entry point; it keeps the local posterior table in a fixed array inside the library instead of
a caller workspace. This test calls it through the C ABI twice in a row (two different noise
levels, so the second call must overwrite the first call's table) and compares every output
with lead_decode's, bit for bit as in the other parity tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_decode_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import workloads
    from paper_2605_17796_gb300 import lead

    inst = workloads.standard("PSL(2,7)", 0)
    code = lead.Code.from_instance(inst).prepare(0)
    info = code.info
    shots = 300
    ex = torch.zeros((shots, info.words_n), dtype=torch.int32, device="cuda")
    sz = torch.zeros((shots, info.words_m[0]), dtype=torch.int32, device="cuda")
    for call, p in enumerate((0.05, 0.02)):
        code.sample(lead.NOISE_X, p, shots, 123 + call, 0, err_x=ex, syn_z=sz)
        o = lead.opts(side=0, p=p)
        ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
        outs = []
        for use_noalloc in (False, True):
            corr = torch.full((shots, info.words_n), -1, dtype=torch.int32, device="cuda")
            st = torch.zeros(shots, dtype=torch.uint8, device="cuda")
            it = torch.full((shots,), -1, dtype=torch.int32, device="cuda")
            llr = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
            if use_noalloc:
                code.decode_noalloc(o, sz, shots, corr, st, it, llr)
            else:
                code.decode(o, sz, shots, corr, st, it, llr, workspace=ws)
            torch.cuda.synchronize()
            outs.append((corr.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy(), llr.cpu().numpy()))
        (c0, s0, i0, l0), (c1, s1, i1, l1) = outs
        assert (c0 == c1).all() and (s0 == s1).all() and (i0 == i1).all()
        assert (l0.view(np.uint32) == l1.view(np.uint32)).all()
        assert (s1 == lead.ST_CONVERGED).any()
