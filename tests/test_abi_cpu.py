"""CPU tests of the C ABI: the library loads, exports every declared symbol, and its host-side
code construction matches the oracle's (no device calls)."""
import os
import re

import numpy as np
import pytest

import workloads
from oracle import tanner

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lead():
    from paper_2605_17796_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    from paper_2605_17796_gb300 import lead as L
    return L


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "lead.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lead_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lead):
    names = _declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lead.LIB, name), name
        assert name in lead.EXPORTS, f"binding lacks {name}"


@pytest.mark.parametrize("name", ["SL(2,3)", "PSL(2,7)"])
def test_host_construction_matches_oracle(lead, name):
    inst = workloads.standard(name, 0)
    code = lead.Code.from_instance(inst)
    oc = tanner.from_instance(inst)
    assert code.info.n == oc.n and code.info.k == oc.k
    assert code.info.rank == (oc.rank_HZ, oc.rank_HX)
    for s in (0, 1):
        assert (code.views(s) == oc.sides[s].views).all()
        assert (code.check_matrix(s) == oc.sides[s].H).all()
        assert code.info.m_l[s] == oc.sides[s].m_l
    assert code.info.prepared_device == -1


def test_paper_local_code_matches_oracle(lead):
    inst = workloads.paper_instance("PSL(2,7)")
    code = lead.Code.from_instance(inst)
    oc = tanner.from_instance(inst)
    for s in (0, 1):
        assert (code.check_matrix(s) == oc.sides[s].H).all()


def test_error_codes(lead):
    inst = workloads.standard("SL(2,3)", 0)
    G = inst.G
    with pytest.raises(lead.LeadError) as e:
        lead.Code(G.mul, inst.A, inst.A, inst.GA)          # B = A: classes shared, TNC fails
    assert e.value.rc == -2
    A = list(inst.A)
    A[0] = G.identity
    with pytest.raises(lead.LeadError) as e:
        lead.Code(G.mul, A, inst.B, inst.GA)
    assert e.value.rc == -3
    bad = G.mul.copy()
    bad[0, 0], bad[0, 1] = bad[0, 1], bad[0, 0]
    with pytest.raises(lead.LeadError) as e:
        lead.Code(bad, inst.A, inst.B, inst.GA)
    assert e.value.rc == -9
    with pytest.raises(lead.LeadError) as e:
        lead.Code(G.mul, inst.A, inst.B, np.zeros((2, 4), dtype=np.uint8))
    assert e.value.rc == -1
    assert b"bounds check" in lead.LIB.lead_status_string(lead.ECHECK)


def test_release_build_is_unchecked(lead):
    """The library the tests load by default is the release build; a code that never failed a
    bounds check reports an all-zero record."""
    assert not lead.CHECKED and lead.LIB.lead_build_flags() == 0
    inst = workloads.standard("SL(2,3)", 0)
    assert lead.Code.from_instance(inst).check_record() == (0, 0, 0, 0)


def test_device_calls_refuse_unprepared_code(lead):
    inst = workloads.standard("SL(2,3)", 0)
    code = lead.Code.from_instance(inst)
    rc = lead.LIB.lead_check(code._h, 0, None, None, 0, None, None)
    assert rc == -8          # LEAD_ESTATE: no device tables


def test_autotune_argument_checks(lead):
    """lead_code_autotune validates its arguments before it touches a device, and refuses a code
    without device tables."""
    code = lead.Code.from_instance(workloads.standard("SL(2,3)", 0))
    for side, prec, p, shots in ((2, 0, 0.05, 64), (0, 3, 0.05, 64), (0, 0, 0.0, 64), (0, 0, 0.5, 64),
                                 (0, 0, 0.05, 0), (1, 1, 0.05, (1 << 24) + 1)):
        assert lead.LIB.lead_code_autotune(code._h, side, prec, p, shots, None, 0) == -1     # LEAD_EINVAL
    assert lead.LIB.lead_code_autotune(None, 0, 0, 0.05, 64, None, 0) == -1
    assert lead.LIB.lead_code_autotune(code._h, 0, 0, 0.05, 64, None, 0) == -8              # LEAD_ESTATE


@pytest.mark.parametrize("name", ["SL(2,3)", "PSL(2,7)"])
def test_min_sum_kernel_specialises_without_a_gpu(lead, name):
    """lead_code_compile runs NVRTC for sm_103a on the host; no device is needed."""
    code = lead.Code.from_instance(workloads.standard(name, 0))
    log = code.compile()
    assert "error" not in log.lower()
    code.compile()        # a second call is a no-op


def test_workspace_sizes_keep_alignment():
    """Workspace sizes are multiples of 256 bytes, so callers can place several workspaces end
    to end (the decode server does, one per side) and keep each 16-byte aligned."""
    from paper_2605_17796_gb300 import lead
    import workloads
    for name in ("SL(2,3)", "PSL(2,7)", "PSL(2,11)"):
        code = lead.Code.from_instance(workloads.standard(name, 0))
        for side in (0, 1):
            for use_lead in (True, False):
                o = lead.opts(side=side, p=0.03, use_lead=use_lead)
                assert code.workspace_bytes(o) % 256 == 0
                assert code.priors_workspace_bytes(o, 1000) % 256 == 0


def test_checked_build_compiles():
    """The checked library builds, reports its flag, and its min-sum kernels (with the bounds
    tests) specialise through NVRTC without a GPU."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-m", "paper_2605_17796_gb300.build", "--checked"], cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    code = ("import workloads\n"
            "from paper_2605_17796_gb300 import lead\n"
            "assert lead.CHECKED and lead.LIB.lead_build_flags() == lead.BUILD_CHECKED\n"
            "for name in ('SL(2,3)', 'PSL(2,7)'):\n"
            "    lead.Code.from_instance(workloads.standard(name, 0)).compile()\n"
            "print('ok')\n")
    env = dict(os.environ, LEAD_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-3000:]


def test_iterated_workspace_size(lead):
    """lead_iterated_workspace_bytes: a multiple of 256 that grows by the compacted batch's
    4 n + 4 words_m + 4 words_n + 9 bytes per shot (up to the 256-byte rounding of each region)
    on top of the decoders' own workspace."""
    inst = workloads.standard("PSL(2,7)", 0)
    code = lead.Code.from_instance(inst)
    info = code.info
    o = lead.opts(side=0, p=0.03)
    per_shot = 4 * info.n + 4 * info.words_m[0] + 4 * info.words_n + 9
    for shots in (1, 1000, 1 << 16):
        total = code.iterated_workspace_bytes(o, shots)
        inner = max(code.workspace_bytes(o, shots), code.priors_workspace_bytes(o, shots))
        assert total % 256 == 0
        extra = total - inner
        assert per_shot * shots <= extra <= per_shot * shots + 8 * 256 + 256
