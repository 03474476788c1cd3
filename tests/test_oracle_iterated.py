"""Oracle pins for iterated LEAD (an extension of Algorithm 1: further rounds on the unconverged
shots, with the last global posterior as per-qubit prior).

What fixes it independently of its own code:
* one round is Algorithm 1 itself;
* a posterior that is strongly signed by a true error e hands every view a prior under which
  e's restriction is by far the most likely local error, so Phases 1-2 return LLRs with e's
  signs and min-sum stops at iteration 0 on e. A flipped sign convention of the conversion
  (probability of no flip instead of a flip) gives the complement instead;
* a zero posterior is the uninformative prior 1/2: every local coset of a linear code with no
  unit vector in its dual is balanced in every position, so q_j = 1/2 exactly, the merge gives
  lambda = 0, and min-sum can never leave the zero decision;
* rounds only touch unconverged shots, converged outputs satisfy H e = s, iterations add up;
* the binary32 conversion p = 1/(1 + e^post) stays within 3 units in the last place of the
  closed form, is monotone, gives exactly 1/2 at 0, and lands beyond the prior clamp outside
  [-17, 17].
"""
import numpy as np
import pytest

from oracle import lead, local, philox


def _shots(code, side_id, p, shots, seed=3):
    noise = philox.NOISE_X if side_id == 0 else philox.NOISE_Z
    x, z = philox.sample_errors(noise, p, seed, np.arange(shots), code.n)
    e = x if side_id == 0 else z
    return e, philox.syndromes(code.sides[side_id].H, e)


def test_one_round_is_algorithm_1(sl3):
    _, code = sl3
    e, syn = _shots(code, 0, 0.06, 60)
    want = lead.decode(code, 0, syn, 0.06)
    got = lead.decode_iterated(code, 0, syn, 0.06, rounds=1)
    for w, g in zip(want, got):
        assert (w.view(np.uint8) == g.view(np.uint8)).all()


@pytest.mark.parametrize("side_id,use_lead", [(0, True), (1, True), (0, False)])
def test_signed_posterior_recovers_the_error(sl3, side_id, use_lead):
    _, code = sl3
    e, syn = _shots(code, side_id, 0.08, 12, seed=5)
    assert e.any(axis=1).all()
    post = np.where(e == 1, np.float32(-20.0), np.float32(20.0)).astype(np.float32)
    corr, st, it, _ = lead.redecode(code, side_id, syn, post, use_lead=use_lead)
    assert (corr == e).all()
    assert (st == lead.STATUS_CONVERGED).all() and (it == 0).all()


def test_zero_posterior_is_uninformative(sl3):
    _, code = sl3
    e, syn = _shots(code, 0, 0.08, 6, seed=7)
    half = local.flip_prob_f32(np.zeros((6, code.n), dtype=np.float32))
    assert (half == np.float32(0.5)).all()
    q, _ = lead.local_priors(code, 0, syn, half)
    assert (q == 0.5).all()
    assert (lead.merge_priors_f32(code, 0, q) == 0).all()
    corr, st, it, post = lead.redecode(code, 0, syn, np.zeros((6, code.n), dtype=np.float32), max_iter=5)
    nz = syn.any(axis=1)
    assert nz.any()
    assert not corr.any()
    assert (st[nz] == lead.STATUS_MAX_ITER).all() and (it[nz] == 5).all()
    assert (st[~nz] == lead.STATUS_CONVERGED).all() and (it[~nz] == 0).all()
    assert (post == 0).all()


def test_rounds_touch_only_unconverged_shots(sl3):
    _, code = sl3
    H = code.sides[0].H
    e, syn = _shots(code, 0, 0.07, 80, seed=11)
    c0, s0, i0, p0 = lead.decode(code, 0, syn, 0.07)
    c3, s3, i3, p3 = lead.decode_iterated(code, 0, syn, 0.07, rounds=3)
    conv0 = s0 == lead.STATUS_CONVERGED
    assert 0 < conv0.sum() < len(conv0)
    assert (c3[conv0] == c0[conv0]).all() and (i3[conv0] == i0[conv0]).all()
    assert (p3[conv0].view(np.uint32) == p0[conv0].view(np.uint32)).all()
    conv3 = s3 == lead.STATUS_CONVERGED
    assert (conv3 | ~conv0).all() and conv3.sum() >= conv0.sum()
    assert (philox.syndromes(H, c3)[conv3] == syn[conv3]).all()
    redo = ~conv0
    assert (i3[redo] >= i0[redo] + np.where(conv3[redo], 0, 32)).all()
    # round 1 of the re-decoded shots is redecode applied to their round-0 posteriors
    c1, s1, i1, _ = lead.redecode(code, 0, syn[redo], p0[redo])
    c2, s2, i2, _ = lead.decode_iterated(code, 0, syn, 0.07, rounds=2)
    assert (c2[redo] == c1).all() and (s2[redo] == s1).all() and (i2[redo] == i0[redo] + i1).all()


def test_flip_probability_binary32():
    x = np.linspace(-17.0, 17.0, 400001).astype(np.float32)
    p = local.flip_prob_f32(x)
    exact = 1.0 / (1.0 + np.exp(x.astype(np.float64)))
    ulp = np.spacing(exact.astype(np.float32)).astype(np.float64)
    assert (np.abs(p.astype(np.float64) - exact) <= 3.0 * ulp).all()
    assert (np.diff(p.astype(np.float64)) <= 0).all()
    assert local.flip_prob_f32(np.float32(0.0)) == np.float32(0.5)
    far = np.array([17.0, 30.0, 1e30, np.inf], dtype=np.float32)
    assert (local.flip_prob_f32(far) < local.P_MIN_F).all()
    assert (local.flip_prob_f32(-far) >= local.P_MAX_F).all()
