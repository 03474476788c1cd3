"""Oracle pins for the code construction (Sec. II): group tables, complex counts, CSS, Appendix A."""
import os

import numpy as np
import pytest

import workloads
from oracle import gf2, tanner

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("name,q,proj", [("SL(2,3)", 3, False), ("PSL(2,7)", 7, True), ("PSL(2,11)", 11, True)])
def test_group_orders_and_axioms(name, q, proj):
    G = workloads.group(name)
    expect = q * (q * q - 1) // (2 if proj else 1)        # |SL(2,q)| = q(q^2-1), PSL halves it
    assert G.order == expect
    n = G.order
    e = G.identity
    assert (G.mul[e] == np.arange(n)).all() and (G.mul[:, e] == np.arange(n)).all()
    assert (G.mul[np.arange(n), G.inv] == e).all()
    rng = np.random.default_rng(1)
    a, b, c = rng.integers(0, n, (3, 2000))
    assert (G.mul[G.mul[a, b], c] == G.mul[a, G.mul[b, c]]).all()


def test_conjugacy_classes_known_counts():
    # SL(2,3) has 7 classes, PSL(2,7) has 6 (orders 1,2,3,4,7,7).
    assert len(set(workloads.conjugacy_class_ids(workloads.group("SL(2,3)")).tolist())) == 7
    assert len(set(workloads.conjugacy_class_ids(workloads.group("PSL(2,7)")).tolist())) == 6


def _check_code(inst, code):
    G = inst.G
    delta = inst.delta
    # Sec. III-C: n = |G| Delta^2 / 2 qubits, |V0| = |G| local decoders of length Delta^2
    assert code.n == G.order * delta * delta // 2
    for side in code.sides:
        assert side.views.shape == (G.order, delta * delta)
        # each vertex sees Delta^2 distinct faces (TNC, Sec. II-A)
        for v in range(G.order):
            assert len(set(side.views[v].tolist())) == delta * delta
        counts = np.bincount(side.views.ravel(), minlength=code.n)
        assert (counts == 2).all()
    # each face has 4 distinct vertices: its two V0 views differ and its two V1 views differ
    qv0 = code.sides[0].qubit_views
    qv1 = code.sides[1].qubit_views
    assert (qv0[:, 0, 0] != qv0[:, 1, 0]).all() and (qv1[:, 0, 0] != qv1[:, 1, 0]).all()
    # CSS condition H_X H_Z^T = 0 (Sec. II-B); binary32 products are exact integers here (each
    # entry counts at most n < 2^24 overlaps)
    prod = np.rint(code.HX.astype(np.float32) @ code.HZ.T.astype(np.float32)).astype(np.int64) % 2
    assert not prod.any()
    # generator weight at most Delta^2
    assert code.HX.sum(axis=1).max() <= delta * delta and code.HZ.sum(axis=1).max() <= delta * delta
    if code.n <= 4096:           # the larger code's ranks are the ones its build computed
        assert code.k == code.n - gf2.rank(code.HX) - gf2.rank(code.HZ)
    assert code.k == code.n - code.rank_HX - code.rank_HZ
    assert code.k >= 1


def test_sl3_instance(sl3):
    inst, code = sl3
    _check_code(inst, code)
    assert code.n == 192


def test_psl11_instance():
    """The seeded PSL(2,11) instance (|G| = 660, Delta = 6): n = 11 880 qubits, CSS, two views per
    qubit and side, k = n - rank H_X - rank H_Z = 2 >= 1."""
    inst = workloads.standard("PSL(2,11)", 0)
    code = tanner.from_instance(inst)
    _check_code(inst, code)
    assert code.n == 11880 and code.k == 2


def test_psl7_instance(psl7):
    inst, code = psl7
    _check_code(inst, code)
    assert code.n == 3024 and code.HZ.shape == (1512, 3024)


def test_paper_local_code_instance():
    inst = workloads.paper_instance("PSL(2,7)")
    code = tanner.from_instance(inst)
    _check_code(inst, code)
    # Sec. IV-B: the printed H_A defines a [6,3,3] code
    GA = workloads.paper_GA()
    assert not ((GA.astype(int) @ workloads.paper_HA().T.astype(int)) % 2).any()
    weights = [int(((np.array([(m >> i) & 1 for i in range(3)]) @ GA) % 2).sum()) for m in range(1, 8)]
    assert min(weights) == 3


def test_views_side1_follow_face_definition(sl3):
    """A V1 vertex h sees at (a, b) a face containing (h,1), (ah,0), (hb,0), (ahb,1)."""
    inst, code = sl3
    G = inst.G
    faces = code.faces
    A, B = inst.A, inst.B
    for h in range(G.order):
        for ia in range(inst.delta):
            for ib in range(inst.delta):
                g, fa, fb = faces[code.sides[1].views[h, ib * inst.delta + ia]]
                a, b = A[fa], B[fb]
                v0 = {int(g), int(G.mul[G.mul[a, g], b])}
                v1 = {int(G.mul[a, g]), int(G.mul[g, b])}
                a2, b2 = A[ia], B[ib]
                assert v1 == {h, int(G.mul[G.mul[a2, h], b2])}
                assert v0 == {int(G.mul[a2, h]), int(G.mul[h, b2])}


def test_tnc_violation_rejected():
    G = workloads.group("SL(2,3)")
    inst = workloads.standard("SL(2,3)", 0)
    with pytest.raises(ValueError):
        tanner.build(G.mul, G.inv, G.identity, inst.A, inst.A, inst.GA)   # B = A shares classes


def test_appendix_a_local_matrix():
    """Appendix A: for C_A = rep-3 and C_B = C_A^perp the X-type local check matrix (our V1 side,
    kron(H_B, H_A) in local order j = b*Delta + a) equals Eq. (product), a [9,7,2] code."""
    rows = np.loadtxt(os.path.join(GOLDEN, "appendix_a_local_matrix.txt"), dtype=np.uint8)
    GA = np.array([[1, 1, 1]], dtype=np.uint8)
    GB = gf2.dual_basis(GA)
    HA = gf2.dual_basis(GA)
    HB = gf2.dual_basis(GB)
    L1 = np.kron(HB, HA)
    assert (gf2.rref(L1)[0] == gf2.rref(rows)[0]).all()
    # and the other order does not reproduce it
    assert not (gf2.rref(np.kron(HA, HB))[0] == gf2.rref(rows)[0]).all()
    ker = gf2.kernel_basis(rows)
    assert ker.shape[0] == 7
    dmin = min(int(((np.array([(m >> i) & 1 for i in range(7)]) @ ker) % 2).sum()) for m in range(1, 128))
    assert dmin == 2
