"""Pins of the OSD oracle (oracle/osd.py) against brute force and the GF(2) rank."""
import itertools

import numpy as np
import pytest

import workloads
from oracle import gf2, lead, osd, philox, tanner


def test_order_keys_follow_float_order():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(5000).astype(np.float32) * 30,
                        np.array([0.0, -0.0, np.inf, -np.inf, 1e-40, -1e-40], dtype=np.float32)])
    k = osd.order_keys(x)
    i = np.argsort(k, kind="stable")
    xs = x[i].astype(np.float64)
    assert np.all(np.diff(xs) >= 0)
    assert osd.order_keys(np.array([-0.0], np.float32))[0] < osd.order_keys(np.array([0.0], np.float32))[0]


def _basis_by_rank(H, order):
    """Pivot positions by rank increments: position c is in S iff adding column order[c] raises
    the rank of the columns before it (an independent route to the elimination's basis)."""
    S, r = [], 0
    for c in range(len(order)):
        rc = gf2.rank(H[:, order[:c + 1]])
        if rc > r:
            S.append(c)
            r = rc
    return S


@pytest.mark.parametrize("seed", range(12))
def test_osd_equals_brute_force_on_small_systems(seed):
    rng = np.random.default_rng(seed)
    m, n, lam = 5, 11, 3
    H = rng.integers(0, 2, size=(m, n)).astype(np.uint8)
    e_true = (rng.random(n) < 0.25).astype(np.uint8)
    s = ((H.astype(np.int64) @ e_true) & 1).astype(np.uint8)
    post = (rng.standard_normal(n) * 3).astype(np.float32)
    prior = (rng.random(n) * 4 - 0.5).astype(np.float32)
    e, idx = osd.osd(H, s, post, prior, lam)
    assert (((H.astype(np.int64) @ e) & 1) == s).all()
    order = osd.column_order(post)
    S = _basis_by_rank(H, order)
    T = [c for c in range(n) if c not in S]
    W = osd.integer_weights(prior)[order]
    fam = [()] + [(c,) for c in T] + list(itertools.combinations(T[:lam], 2))
    best = None
    for ci, flips in enumerate(fam):
        # the unique solution with these T columns set (S is a basis): search all solutions
        sols = []
        for bits in itertools.product((0, 1), repeat=n):
            eo = np.array(bits, dtype=np.uint8)
            if [c for c in T if eo[c]] != list(flips):
                continue
            e_q = np.zeros(n, dtype=np.uint8)
            e_q[order] = eo
            if (((H.astype(np.int64) @ e_q) & 1) == s).all():
                sols.append((int((eo.astype(np.int64) * W).sum()), e_q))
        assert len(sols) == 1
        if best is None or sols[0][0] < best[0]:
            best = (sols[0][0], ci, sols[0][1])
    assert idx == best[1]
    assert (e == best[2]).all()


def test_osd_outputs_satisfy_the_syndrome(sl3):
    inst, code = sl3
    H = code.sides[0].H
    x, _ = philox.sample_errors(philox.NOISE_X, 0.08, 4, np.arange(40), code.n)
    syn = philox.syndromes(H, x)
    lam = lead.prior_f32(code, 0, syn, 0.08)
    _, _, _, post = lead.min_sum(H, code.sides[0].m_l, syn, lam, 32)
    corr, idx = osd.osd_batch(H, syn, post, lam, 3)
    assert (philox.syndromes(H, corr) == syn).all()
    assert (idx >= 0).all()


def test_osd0_recovers_a_low_weight_error_on_reliable_positions(psl7):
    """If the posterior marks exactly the error's qubits as most likely flipped and the error's
    columns are independent, OSD-0 returns that error (its columns lead the basis)."""
    inst, code = psl7
    H = code.sides[0].H
    rng = np.random.default_rng(3)
    e = np.zeros(code.n, dtype=np.uint8)
    e[rng.choice(code.n, 4, replace=False)] = 1
    assert gf2.rank(H[:, e == 1]) == 4
    s = ((H.astype(np.int64) @ e) & 1).astype(np.uint8)
    post = np.where(e == 1, -5.0, 5.0).astype(np.float32)
    prior = np.full(code.n, 3.0, dtype=np.float32)
    got, idx = osd.osd(H, s, post, prior, 0)
    assert idx == 0 and (got == e).all()
