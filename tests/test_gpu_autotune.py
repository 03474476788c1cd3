"""lead_code_autotune: the min-sum kernel (Algorithm 1, Phase 3) kept after timing several
launch shapes (shots per CTA or cluster size, register cap) decodes every shot bit-identically
to the default kernel, in each precision mode, at the tuned prior and at another one it
serves, and the report names one kept candidate per call."""
import numpy as np
import pytest

import workloads
from oracle import philox, tanner

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2605_17796_gb300 import lead
    return lead


def _decode(L, code, side, syn_dev, shots, p, precision):
    info = code.info
    o = L.opts(side=side, p=p, precision=precision)
    ws = torch.zeros(code.workspace_bytes(o) // 4 + 64, dtype=torch.int32, device="cuda")
    corr = torch.zeros((shots, info.words_n), dtype=torch.int32, device="cuda")
    st = torch.zeros(shots, dtype=torch.uint8, device="cuda")
    it = torch.zeros(shots, dtype=torch.int32, device="cuda")
    post = torch.zeros((shots, info.n), dtype=torch.float32, device="cuda")
    code.decode(o, syn_dev, shots, corr, st, it, llr=post, workspace=ws)
    torch.cuda.synchronize()
    return corr.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy(), post.cpu().numpy()


@pytest.mark.parametrize("name,side,p,shots", [("SL(2,3)", 1, 0.06, 300), ("PSL(2,7)", 0, 0.05, 200),
                                               ("PSL(2,11)", 1, 0.025, 12)])
def test_tuned_kernel_is_bit_identical(L, name, side, p, shots):
    inst = workloads.standard(name, 0)
    oc = tanner.from_instance(inst)
    x, z = philox.sample_errors(philox.NOISE_DEPOL, 1.5 * p, 5, np.arange(shots), oc.n)
    e = x if side == 0 else z
    syn = philox.syndromes(oc.sides[side].H, e)
    for precision in (0, 1, 2):
        code = L.Code.from_instance(inst).prepare(0)
        dev = torch.from_numpy(philox.pack_bits(syn, code.info.words_m[side]).view(np.int32)).cuda()
        # decodes at p and at p / 2 (which the shape tuned at p also serves: the nearest tuned p)
        before = [_decode(L, code, side, dev, shots, q, precision) for q in (p, p / 2)]
        report = code.autotune(side, precision, p, shots=min(4096, 64 * shots))
        print(f"{name} side {side} precision {precision}:\n{report}")
        assert report.count("<- kept") == 1
        after = [_decode(L, code, side, dev, shots, q, precision) for q in (p, p / 2)]
        for bq, aq in zip(before, after):
            for a, b in zip(bq, aq):
                assert a.dtype == b.dtype and (a == b).all()
        assert code.device_errors() == 0
