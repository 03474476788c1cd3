"""Oracle pins for the sampler (Philox4x32-10, noise models) and Algorithm 1's merge and min-sum."""
import itertools
import os

import numpy as np
import pytest

from oracle import lead, local, philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_published_vectors():
    """Known-answer vectors of Philox4x32-10 published with the Random123 library (SC'11)."""
    vecs = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
            ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
            ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
             (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for c, k, want in vecs:
        out = philox.philox4x32_10(*[np.array([x], dtype=np.uint64) for x in c], *k)
        assert tuple(int(o[0]) for o in out) == want


def test_counter_based_shot_offsets():
    u_all = philox.uniforms(1234, np.arange(20), 50)
    u_sub = philox.uniforms(1234, np.arange(7, 11), 50)
    assert (u_all[7:11] == u_sub).all()
    big = philox.uniforms(5, np.array([2 ** 40 + 3]), 10)
    assert big.shape == (1, 10) and not (big == philox.uniforms(5, np.array([3]), 10)).all()


def _wilson_contains(k, n, p, z=4.5):
    ph = k / n
    den = 1 + z * z / n
    c = (ph + z * z / (2 * n)) / den
    h = z * np.sqrt(ph * (1 - ph) / n + z * z / (4 * n * n)) / den
    return c - h <= p <= c + h


def test_bernoulli_and_depolarizing_frequencies():
    n, S = 3024, 100
    x, z = philox.sample_errors(philox.NOISE_X, 0.05, 7, np.arange(S), n)
    assert not z.any() and _wilson_contains(int(x.sum()), n * S, 0.05)
    x, z = philox.sample_errors(philox.NOISE_DEPOL, 0.09, 7, np.arange(S), n)
    X = x & (1 - z)
    Y = x & z
    Z = z & (1 - x)
    for part in (X, Y, Z):
        assert _wilson_contains(int(part.sum()), n * S, 0.03)


def test_thresholds_exact():
    tb, (t1, t2, t3) = philox.thresholds(0.05)
    assert tb == int(np.floor(0.05 * 2 ** 32)) == t3
    assert t1 <= t2 <= t3 and abs(t2 - 2 * t1) <= 1


def test_pack_roundtrip():
    rng = np.random.default_rng(3)
    b = rng.integers(0, 2, (5, 100)).astype(np.uint8)
    w = philox.pack_bits(b, 4)
    assert (philox.unpack_bits(w, 100) == b).all()
    assert (w[:, 3] >> 4 == 0).all()       # padding bits stay zero


def test_appendix_a_merge():
    """Appendix A, Phase 2 worked example: alpha * Average({0.21, 0.25}) = 0.23."""
    q1, q2, alpha, want = np.loadtxt(os.path.join(GOLDEN, "appendix_a_merge.txt"))
    assert abs(lead.merge_f64(q1, q2, alpha) - want) < 1e-15
    assert abs(lead.merge_f64(q1, q2, 0.01) - 0.0023) < 1e-15


def _tree_code(n_checks, rng):
    """A random tree on the checks; every tree edge is a qubit in two checks, plus pendant qubits
    in one check. Its Tanner graph is cycle-free."""
    edges = [(int(rng.integers(0, c)), c) for c in range(1, n_checks)]
    cols = []
    for a, b in edges:
        col = np.zeros(n_checks, dtype=np.uint8)
        col[a] = col[b] = 1
        cols.append(col)
    deg = np.zeros(n_checks, dtype=int)
    for a, b in edges:
        deg[a] += 1
        deg[b] += 1
    for c in range(n_checks):
        # pendant qubits; every check keeps degree >= 2 (a degree-1 check would send an
        # infinite message, which never happens on the codes decoded here)
        for _ in range(max(int(rng.integers(0, 2)), 2 - int(deg[c]))):
            col = np.zeros(n_checks, dtype=np.uint8)
            col[c] = 1
            cols.append(col)
    return np.array(cols, dtype=np.uint8).T


def test_min_sum_is_exact_ml_on_a_tree():
    """Textbook special case: on a cycle-free Tanner graph min-sum (max-product) finds the
    maximum-likelihood error, i.e. the solution of H e = s of least total LLR weight, once the
    messages have travelled the whole tree (run without early stopping)."""
    rng = np.random.default_rng(11)
    trials = 0
    for _ in range(30):
        H = _tree_code(int(rng.integers(4, 8)), rng)
        m, n = H.shape
        if n > 14:
            continue
        lam = rng.uniform(0.3, 4.0, (1, n)).astype(np.float32)
        allv = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.uint8)
        syns = (allv.astype(int) @ H.T.astype(int)) % 2
        for _ in range(4):
            e = rng.integers(0, 2, n).astype(np.uint8)
            s = ((H.astype(int) @ e) % 2).astype(np.uint8)
            sel = allv[(syns == s).all(axis=1)]
            cost = sel.astype(np.float64) @ lam[0].astype(np.float64)
            if np.sort(cost)[1] - cost.min() < 1e-3:
                continue                      # ML not unique; skip
            ml = sel[np.argmin(cost)]
            corr, st, it, _ = lead.min_sum(H, 1, s[None, :], lam, max_iter=2 * m, early_stop=False)
            assert st[0] == lead.STATUS_CONVERGED
            assert (corr[0] == ml).all()
            trials += 1
    assert trials > 20


def test_zero_syndrome_gives_zero_correction(psl7):
    inst, code = psl7
    syn = np.zeros((3, code.HZ.shape[0]), dtype=np.uint8)
    for use_lead in (True, False):
        corr, st, it, _ = lead.decode(code, 0, syn, 0.05, use_lead=use_lead)
        assert not corr.any() and (st == lead.STATUS_CONVERGED).all() and (it == 0).all()


def test_converged_outputs_satisfy_syndrome(sl3):
    inst, code = sl3
    for side_id, noise in ((0, philox.NOISE_X), (1, philox.NOISE_Z)):
        x, z = philox.sample_errors(noise, 0.04, 3, np.arange(300), code.n)
        e = x if side_id == 0 else z
        H = code.sides[side_id].H
        syn = philox.syndromes(H, e)
        corr, st, it, _ = lead.decode(code, side_id, syn, 0.04)
        conv = st == lead.STATUS_CONVERGED
        assert conv.mean() > 0.5
        assert (philox.syndromes(H, corr)[conv] == syn[conv]).all()
        f = lead.check(code, side_id, e, corr)
        assert ((f & 1) == 0)[conv].all()
        assert ((f & 1) == 1)[~conv].all()


def test_check_flags_logicals(sl3):
    """A residual in ker H_Z outside rowspace H_X is flagged as a logical error; a stabilizer is not."""
    inst, code = sl3
    from oracle import gf2
    kerZ = gf2.kernel_basis(code.HZ)
    rs = gf2.RowSpace(code.HX)
    logical = next(v for v in kerZ if not rs.contains(v))
    stab = code.HX[0]
    zero = np.zeros((2, code.n), dtype=np.uint8)
    f = lead.check(code, 0, zero, np.stack([logical, stab]))
    assert list(f) == [2, 0]


def test_prior_f32_close_to_f64(psl7):
    inst, code = psl7
    x, _ = philox.sample_errors(philox.NOISE_X, 0.03, 0, np.arange(20), code.n)
    syn = philox.syndromes(code.HZ, x)
    _, l64 = lead.prior_f64(code, 0, syn, 0.03)
    l32 = lead.prior_f32(code, 0, syn, 0.03)
    assert np.abs(l64 - l32.astype(np.float64)).max() < 1e-4


def _nearest_even(x, keep_bits):
    """Brute force in binary64: the two binary32 values whose patterns end in 32-keep_bits zero
    bits around x, and the nearer one (ties: the one whose kept pattern is even)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.int64)
    drop = 32 - keep_bits
    lo = (u >> drop) << drop
    hi = lo + (1 << drop)
    flo = lo.astype(np.uint32).view(np.float32).astype(np.float64)
    fhi = hi.astype(np.uint32).view(np.float32).astype(np.float64)
    xv = np.asarray(x, dtype=np.float32).astype(np.float64)
    dlo, dhi = np.abs(xv - flo), np.abs(fhi - xv)
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (((lo >> drop) & 1) == 1))
    return np.where(pick_hi, fhi, flo).astype(np.float32)


def test_bf16_rounding_is_nearest_even():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * np.float32(30),
                        rng.standard_normal(2000).astype(np.float32) * np.float32(1e-39),   # subnormal
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0, -0.0],
                                 dtype=np.float32)])
    got = lead.round_bf16(x)
    want = _nearest_even(np.abs(x), 16) * np.sign(x).astype(np.float32)
    assert (got[x != 0] == want[x != 0]).all()
    assert list(got[-5:-2]) == [1.0, 1.0 + 2 ** -6, -1.0]               # ties to the even pattern
    assert np.signbit(got[-1]) and not np.signbit(got[-2])
    assert not (got.view(np.uint32) & 0xFFFF).any()                      # bfloat16 patterns


def test_storage_rounding_modes():
    x = np.array([0.1, -3.3, 1000.5, 1e-8], dtype=np.float32)
    assert (lead.round_storage(x, lead.PREC_FP32) == x).all()
    assert (lead.round_storage(x, lead.PREC_FP16) == x.astype(np.float16).astype(np.float32)).all()
    big = np.array([7e4, -1e6, 65519.0, 65520.0], dtype=np.float32)
    assert list(lead.round_storage(big, lead.PREC_FP16)) == [65504.0, -65504.0, 65504.0, 65504.0]
    b = lead.round_storage(x, lead.PREC_BF16)
    assert np.all(np.abs(b - x) <= np.abs(x) * 2.0 ** -9)


@pytest.mark.parametrize("precision", [1, 2])
def test_reduced_precision_min_sum(sl3, precision):
    """16-bit storage: zero syndrome still decodes to zero at iteration 0; every converged output
    satisfies H e = s; every posterior returned is a value of the storage format; and the
    failure rate stays that of binary32 storage within sampling noise (the decisions themselves
    differ on shots where min-sum oscillates without converging)."""
    inst, code = sl3
    syn0 = np.zeros((2, code.HZ.shape[0]), dtype=np.uint8)
    corr, st, it, _ = lead.decode(code, 0, syn0, 0.04, precision=precision)
    assert not corr.any() and (st == lead.STATUS_CONVERGED).all() and (it == 0).all()
    x, _ = philox.sample_errors(philox.NOISE_X, 0.03, 5, np.arange(400), code.n)
    syn = philox.syndromes(code.HZ, x)
    corr, st, it, post = lead.decode(code, 0, syn, 0.03, precision=precision)
    conv = st == lead.STATUS_CONVERGED
    assert (philox.syndromes(code.HZ, corr)[conv] == syn[conv]).all()
    assert (lead.round_storage(post, precision) == post).all()
    c32, st32, _, _ = lead.decode(code, 0, syn, 0.03)
    f16 = (lead.check(code, 0, x, corr) != 0).mean()
    f32 = (lead.check(code, 0, x, c32) != 0).mean()
    assert abs(f16 - f32) < 4 * np.sqrt(f32 * (1 - f32) / len(x)) + 0.01
