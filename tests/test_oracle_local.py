"""Oracle pins for the exact local estimator (Phase 1 of Algorithm 1)."""
import math

import numpy as np
import pytest

from oracle import local


def test_delta4_tables_equal_brute_force(sl3):
    inst, code = sl3
    for side in code.sides:
        N, N1, ml = local.tables(side.RA, side.RB)
        Nb, N1b, mlb = local.brute_force(side.L, inst.delta)
        assert (N == Nb).all() and (N1 == N1b).all() and (ml == mlb).all()
        Nr, N1r = local.row_tables(side.RA, side.RB)
        assert (N == Nr).all() and (N1 == N1r).all()


def test_delta4_posterior_equals_defining_sum(sl3):
    inst, code = sl3
    side = code.sides[0]
    N, N1, _ = local.tables(side.RA, side.RB)
    for p in (0.02, 0.05, 0.2):
        q = local.posterior_from_tables(N, N1, p)
        for s in (0, 1, 5, 11, 15):
            qb = local.posterior_brute_force(side.L, s, np.full(16, p))
            assert np.abs(q[s] - qb).max() < 1e-13


@pytest.mark.slow
def test_delta6_fourier_equals_row_grouping(psl7):
    inst, code = psl7
    side = code.sides[0]
    N, N1, _ = local.tables(side.RA, side.RB)
    Nr, N1r = local.row_tables(side.RA, side.RB)
    assert (N == Nr).all() and (N1 == N1r).all()


@pytest.mark.parametrize("side_id", [0, 1])
def test_delta6_closed_forms(psl7, side_id):
    inst, code = psl7
    side = code.sides[side_id]
    N, N1, ml = local.tables(side.RA, side.RB)
    n_l, m_l = 36, side.m_l
    assert m_l == 9
    # every coset has 2^(n_l - m_l) members; all cosets together hold C(n_l, w) patterns of weight w
    assert (N.sum(axis=1) == 2 ** (n_l - m_l)).all()
    assert [int(x) for x in N.sum(axis=0)] == [math.comb(n_l, w) for w in range(n_l + 1)]
    # patterns with e_j = 1 of weight w: C(n_l - 1, w - 1) over all cosets, for every j
    tot = N1.sum(axis=0)
    for j in range(n_l):
        assert [int(x) for x in tot[j]] == [0] + [math.comb(n_l - 1, w - 1) for w in range(1, n_l + 1)]
    # sum_j N1 = w N (each member of weight w has w ones)
    assert (N1.sum(axis=1) == N * np.arange(n_l + 1)[None, :]).all()
    # MacWilliams on the zero coset (the local code itself)
    assert (local.macwilliams_zero_coset(side.L) == N[0]).all()
    # the ML decision lies in the coset and has the least weight present in it
    bits = (ml[:, None] >> np.arange(n_l)[None, :]) & 1
    syn = ((bits @ side.L.T.astype(np.int64)) & 1) @ (1 << np.arange(m_l))
    assert (syn == np.arange(1 << m_l)).all()
    assert (bits.sum(axis=1) == np.argmax(N > 0, axis=1)).all()


def _coset_brute_force(L, s, delta):
    """Enumerate the 2^(n_l - m_l) coset members of syndrome s: weight histogram, per-bit
    histogram of one position, and the least (weight, row-major key) member."""
    from oracle import gf2
    m_l, n_l = L.shape
    ker = gf2.kernel_basis(L)
    R, piv = gf2.rref(L)
    # a particular solution: solve L e = s through the RREF of [L | s]
    aug = np.concatenate([L, np.array([(s >> r) & 1 for r in range(m_l)], dtype=np.uint8)[:, None]], axis=1)
    Ra, pa = gf2.rref(aug)
    e0 = np.zeros(n_l, dtype=np.uint8)
    for i, c in enumerate(pa):
        e0[c] = Ra[i, -1]
    # convert local index j = b*Delta + a to row-major key bit a*Delta + b, as 64-bit ints
    perm = np.array([(j % delta) * delta + (j // delta) for j in range(n_l)])

    def as_key(v):
        return int(sum(int(v[j]) << int(perm[j]) for j in range(n_l)))

    kvec = np.array([as_key(k) for k in ker], dtype=np.uint64)
    x0 = np.uint64(as_key(e0))
    h = kvec.size // 2
    lo = np.zeros(1, dtype=np.uint64)
    for k in kvec[:h]:
        lo = np.concatenate([lo, lo ^ k])
    hi = np.zeros(1, dtype=np.uint64)
    for k in kvec[h:]:
        hi = np.concatenate([hi, hi ^ k])
    hist = np.zeros(n_l + 1, dtype=np.int64)
    best = (n_l + 1, None)
    for c in range(0, lo.size, 256):
        X = (lo[c:c + 256, None] ^ hi[None, :] ^ x0).ravel()
        w = np.bitwise_count(X).astype(np.int64)
        hist += np.bincount(w, minlength=n_l + 1)
        wm = int(w.min())
        if wm <= best[0]:
            cand = int(X[w == wm].min())
            if wm < best[0] or cand < best[1]:
                best = (wm, cand)
    return hist, best


@pytest.mark.slow
def test_delta6_coset_brute_force_sampled(psl7):
    inst, code = psl7
    side = code.sides[0]
    N, N1, ml = local.tables(side.RA, side.RB)
    delta = inst.delta
    for s in (0, 77, 300, 511):
        hist, (wbest, key) = _coset_brute_force(side.L, s, delta)
        assert (hist == N[s]).all()
        # ML mask (local order) -> row-major key
        m = int(ml[s])
        k2 = sum(((m >> j) & 1) << ((j % delta) * delta + j // delta) for j in range(36))
        assert wbest == bin(m).count("1") and key == k2


def test_posterior_small_p_limit(psl7):
    """p -> 0: the posterior is uniform over the least-weight coset members."""
    inst, code = psl7
    side = code.sides[0]
    N, N1, _ = local.tables(side.RA, side.RB)
    q = local.posterior_from_tables(N, N1, 1e-9)
    wmin = np.argmax(N > 0, axis=1)
    lim = N1[np.arange(512), :, wmin] / N[np.arange(512), wmin][:, None]
    assert np.abs(q - lim).max() < 1e-6


def test_posterior_fourier_form_fp64(psl7):
    """Dual-domain closed form of the marginal in FP64 (well conditioned at p = 0.2)."""
    inst, code = psl7
    side = code.sides[0]
    L = side.L.astype(np.int64)
    N, N1, _ = local.tables(side.RA, side.RB)
    p = 0.2
    q = local.posterior_from_tables(N, N1, p)
    rho = 1 - 2 * p
    us = np.arange(512)
    ub = (us[:, None] >> np.arange(9)[None, :]) & 1
    C = (ub @ L) & 1
    for s in (3, 100, 400):
        sg = (-1.0) ** (np.bitwise_count((us & s).astype(np.uint64)).astype(np.int64) & 1)
        T = (sg * rho ** C.sum(axis=1)).sum()
        for j in (0, 17, 35):
            Tj = (sg * rho ** (C.sum(axis=1) + 1 - 2 * C[:, j])).sum()
            assert abs((1 - Tj / T) / 2 - q[s, j]) < 1e-12


def _f32_round_exact(x, Fraction):
    """Binary32 nearest (ties to even) to the rational x, by exact comparison with the midpoints
    of its two binary32 neighbours."""
    est = np.float32(float(x))
    cands = [np.nextafter(est, np.float32(-np.inf), dtype=np.float32), est,
             np.nextafter(est, np.float32(np.inf), dtype=np.float32)]
    dist = [abs(Fraction(float(c)) - x) for c in cands]
    best = min(range(3), key=lambda k: (dist[k], int(cands[k].view(np.uint32)) & 1))
    return cands[best]


def test_llr_f32_is_the_rounded_exact_value():
    """lambda(p) = ln((1-p)/p) rounded to binary32, checked against ln(1-p) - ln(p) evaluated at
    60 digits by mpmath (another identity and another library than the oracle's) and rounded by
    exact rational comparison, on log-uniform p over the clamp range, p near 1/2 and near 2^-23."""
    mpmath = pytest.importorskip("mpmath")
    from fractions import Fraction
    mpmath.mp.dps = 60
    rng = np.random.default_rng(12)
    p = np.concatenate([np.exp2(rng.uniform(-23, -1, 1500)),
                        0.5 - np.exp2(rng.uniform(-24, -3, 400)),
                        np.float32(2.0 ** -23) * (1 + rng.integers(0, 4096, 100).astype(np.float64) * 2.0 ** -23),
                        [2.0 ** -23, 0.25, 0.5, 0.125, 0.01, 0.05]]).astype(np.float32)
    got = local.llr_f32(p)
    for pi, gi in zip(p, got):
        mp = mpmath.mpf(float(pi))
        exact = mpmath.log(1 - mp) - mpmath.log(mp)
        want = _f32_round_exact(Fraction(mpmath.nstr(exact, 55, min_fixed=-100, max_fixed=100)), Fraction)
        assert gi.view(np.uint32) == want.view(np.uint32), (float(pi), float(gi), float(want))


def test_llr_f32_exact_fallback_matches_mpmath():
    """The decimal fallback the oracle uses near rounding boundaries gives the same rounding as
    mpmath's logarithm, on random inputs (it is exercised here directly, since boundary cases
    are rare)."""
    mpmath = pytest.importorskip("mpmath")
    from fractions import Fraction
    mpmath.mp.dps = 60
    rng = np.random.default_rng(13)
    for pi in np.exp2(rng.uniform(-23, -1, 200)).astype(np.float32):
        mp = mpmath.mpf(float(pi))
        exact = mpmath.log((1 - mp) / mp)
        want = _f32_round_exact(Fraction(mpmath.nstr(exact, 55, min_fixed=-100, max_fixed=100)), Fraction)
        assert local._llr_exact_round(pi).view(np.uint32) == want.view(np.uint32)


def test_llr_f32_symmetry_and_fixed_values():
    """lambda(1/2) = 0; lambda(1 - p) = -lambda(p) exactly (1 - p is exact for p > 1/2);
    lambda(1/4) = ln 3 and lambda(2^-k) = ln(2^k - 1) rounded; strictly decreasing on a grid;
    the clamp maps p <= 0 and p >= 1 to the ends of [2^-23, 1 - 2^-23]."""
    assert local.llr_f32(np.array([0.5], dtype=np.float32))[0] == 0.0
    s = np.linspace(0.5, 1 - 2.0 ** -23, 1001)[1:].astype(np.float32)
    assert (local.llr_f32(s) == -local.llr_f32((np.float32(1) - s).astype(np.float32))).all()
    assert local.llr_f32(np.array([0.25], dtype=np.float32))[0] == np.float32(np.log(3.0))
    for k in (1, 2, 5, 10, 20, 23):
        assert local.llr_f32(np.array([2.0 ** -k], dtype=np.float32))[0] == np.float32(np.log(2.0 ** k - 1.0))
    g = np.geomspace(2.0 ** -23, 1 - 2.0 ** -23, 100001).astype(np.float32)
    g = np.unique(g)
    assert (np.diff(local.llr_f32(g).astype(np.float64)) < 0).all()
    ends = local.llr_f32(np.array([0.0, -1.0, 1.0, 2.0], dtype=np.float32))
    lo, hi = local.llr_f32(np.array([2.0 ** -23, 1 - 2.0 ** -23], dtype=np.float32))
    assert (ends == np.array([lo, lo, hi, hi], dtype=np.float32)).all()


def test_boost_applies_to_ml_bits(psl7):
    inst, code = psl7
    side = code.sides[0]
    N, N1, ml = local.tables(side.RA, side.RB)
    lut = local.boosted_table_f32(N, N1, ml, 0.05)
    q = local.posterior_from_tables(N, N1, 0.05).astype(np.float32)
    flip = ((ml[:, None] >> np.arange(36)[None, :]) & 1).astype(bool)
    assert (lut[flip] >= 0.5).all()
    assert (lut[~flip] == q[~flip]).all()


def test_nonuniform_posterior_equals_defining_sum(sl3):
    inst, code = sl3
    rng = np.random.default_rng(5)
    for side in code.sides:
        for s in (0, 3, 9, 15):
            p = rng.uniform(0.01, 0.3, 16)
            got = local.posterior_nonuniform(side.RA, side.RB, s, p)
            want = local.posterior_brute_force(side.L, s, p)
            assert np.abs(got - want).max() < 1e-13


def test_nonuniform_reduces_to_uniform(psl7):
    inst, code = psl7
    side = code.sides[0]
    N, N1, ml = local.tables(side.RA, side.RB)
    q = local.posterior_from_tables(N, N1, 0.04)
    W = local.integer_costs(np.full(36, 0.04))
    for s in (0, 5, 77, 300, 511):
        got = local.posterior_nonuniform(side.RA, side.RB, s, np.full(36, 0.04))
        assert np.abs(got - q[s]).max() < 1e-12
        assert local.ml_nonuniform(side.RA, side.RB, s, W) == int(ml[s])


def test_nonuniform_ml_is_least_cost_brute_force(sl3):
    inst, code = sl3
    side = code.sides[0]
    rng = np.random.default_rng(9)
    es = np.arange(1 << 16)
    bits = ((es[:, None] >> np.arange(16)[None, :]) & 1)
    syn = ((bits @ side.L.T.astype(np.int64)) & 1) @ (1 << np.arange(side.m_l))
    for _ in range(20):
        p = rng.uniform(0.005, 0.4, 16)
        W = local.integer_costs(p)
        s = int(rng.integers(0, 1 << side.m_l))
        sel = es[syn == s]
        cost = bits[syn == s] @ W
        # least cost, ties by the row-major key (local j = b*Delta + a -> key bit a*Delta + b)
        key = sum(((sel >> (b * 4 + a)) & 1) << (a * 4 + b) for a in range(4) for b in range(4))
        want = int(sel[np.lexsort((key, cost))[0]])
        assert local.ml_nonuniform(side.RA, side.RB, s, W) == want


def test_exp_series_f64_accuracy():
    x = np.concatenate([np.linspace(-88.0, 88.0, 400001), [0.0, 1.0, -1.0, np.log(2.0)]])
    got = local.exp_series_f64(x)
    ref = np.exp(x)
    assert np.abs(got - ref).max() <= 4.5e-16 * np.abs(ref).max() or np.all(np.abs(got / ref - 1) <= 4.5e-16)
    assert local.exp_series_f64(np.array([0.0]))[0] == 1.0


def test_sigmoid_inverts_the_prior_llr():
    """sigmoid(lambda(p)) = p: the binary32 LLR of p maps back to p within the LLR's error."""
    p = np.geomspace(1e-4, 0.49, 2001).astype(np.float32)
    q = local.sigmoid_f32(local.llr_f32(p)).astype(np.float64)
    assert np.all(np.abs(q - p) <= 3e-5 * p)
    assert local.sigmoid_f32(np.array([0.0], dtype=np.float32))[0] == np.float32(0.5)
    assert local.sigmoid_f32(np.array([1e4], dtype=np.float32))[0] > 0           # clamp at 88: no underflow to 0


@pytest.mark.parametrize("side_id", [0, 1])
def test_local_minsum_tables(psl7, side_id):
    """The local min-sum estimator: iteration 0 decides the zero syndrome with q = sigmoid(lambda)
    = p; every converged decision satisfies its local syndrome and carries the boost; a table
    with max_iter = 0 is the prior everywhere; more iterations never undo convergence."""
    from oracle import lead
    inst, code = psl7
    side = code.sides[side_id]
    p = 0.04
    q, iters, conv, dec = lead.local_minsum_tables(side.RA, side.RB, p)
    lam = local.llr_f32(np.array([p], dtype=np.float32))[0]
    assert conv[0] and iters[0] == 0 and not dec[0].any()
    assert (q[0] == local.sigmoid_f32(np.array([lam]))[0]).all()
    H = np.kron(side.RB, side.RA).astype(np.int64)
    s_of = ((dec.astype(np.int64) @ H.T) & 1) @ (1 << np.arange(H.shape[0]))
    assert (s_of[conv] == np.arange(len(conv))[conv]).all()
    assert (q[conv][dec[conv] == 1] >= 0.5).all()
    assert iters.max() <= inst.delta ** 2
    q0, it0, conv0, _ = lead.local_minsum_tables(side.RA, side.RB, p, max_iter=0)
    assert (it0 == 0).all() and conv0.sum() == 1 and (q0[1:] == q[0, 0]).all()
