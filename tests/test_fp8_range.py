"""Why the per-qubit-prior contraction keeps two bfloat16 terms rather than FP8 (e4m3).

The marginal contraction's operand W = 2^(score - max) spans tens of binades within one item's
local coset, while e4m3 covers about 17 (normal and subnormal). This test measures, on PSL(2,7)
items with per-qubit priors p_i ~ U[0.015, 0.045] and with the oracle's FP64 row log-sums, the
span of the coset scores and the error of q when W is carried as two e4m3 terms (scaled so that
the largest W is 256), against the same contraction in FP64: the FP8 form misses the 1e-4 bar by
orders of magnitude, while two bfloat16 terms (what the tensor-core kernel uses) stay within it.
"""
import numpy as np

import workloads
from oracle import lead as olead
from oracle import local, philox, tanner


def _round_e4m3(x):
    """Nearest e4m3 value (3 fraction bits, exponents -6 .. 8, subnormals down to 2^-9, largest
    448), ties to even; x >= 0."""
    a = np.minimum(np.asarray(x, dtype=np.float64), 448.0)
    e = np.maximum(np.floor(np.log2(np.maximum(a, 1e-300))), -6.0)
    q = 2.0 ** (e - 3)
    return np.minimum(np.round(a / q) * q, 448.0)


def _round_bf16(x):
    return olead.round_bf16(np.asarray(x, dtype=np.float32)).astype(np.float64)


def _q(F, R, Rb, W, delta, kB):
    Z = W.sum()
    q = np.zeros((delta, delta))
    for a in range(delta):
        agg = np.zeros(1 << kB)
        np.add.at(agg, F[a], W)
        for b in range(delta):
            q[a, b] = (agg * Rb[a, b] / R[a]).sum() / Z
    return q


def test_fp8_cannot_carry_the_coset_weights():
    oc = tanner.from_instance(workloads.standard("PSL(2,7)", 0))
    side = oc.sides[0]
    delta, kB = 6, side.RB.shape[0]
    prior = workloads.per_qubit_priors(2, oc.n, 0.03, 0.5, 5)
    syn = philox.syndromes(side.H, workloads.errors_from_priors(prior, 5))
    sv = olead.local_syndromes(side, syn)
    f_of_x, _, bits, _, _ = local._row_tables(side.RB)
    spans, err8, err16 = [], 0.0, 0.0
    for s in range(prior.shape[0]):
        for v in range(0, side.views.shape[0], 7):
            P = prior[s, side.views[v]].astype(np.float64).reshape(delta, delta).T
            odds = P / (1 - P)
            R = np.zeros((delta, 1 << kB))
            Rb = np.zeros((delta, delta, 1 << kB))
            for a in range(delta):
                w = np.prod(np.where(bits == 1, odds[a][None, :], 1.0), axis=1)
                np.add.at(R[a], f_of_x, w)
                for b in range(delta):
                    sel = bits[:, b] == 1
                    np.add.at(Rb[a, b], f_of_x[sel], w[sel])
            F = local.coset_row_images(side.RA, side.RB, int(sv[s, v]))
            L = np.sum(np.log2(np.stack([R[a][F[a]] for a in range(delta)])), axis=0)
            spans.append(L.max() - L.min())
            W = 2.0 ** (L - L.max())
            q = _q(F, R, Rb, W, delta, kB)
            t1 = _round_e4m3(256.0 * W)
            W8 = (t1 + _round_e4m3(256.0 * W - t1)) / 256.0
            h = _round_bf16(W)
            W16 = h + _round_bf16(W - h)
            err8 = max(err8, float((np.abs(_q(F, R, Rb, W8, delta, kB) - q) / q).max()))
            err16 = max(err16, float((np.abs(_q(F, R, Rb, W16, delta, kB) - q) / q).max()))
    print(f"{len(spans)} items: coset score span median {np.median(spans):.1f} binades, max {max(spans):.1f}; "
          f"largest relative error of q: two e4m3 terms {err8:.2e}, two bfloat16 terms {err16:.2e}")
    assert np.median(spans) > 17
    assert err8 > 1e-3
    assert err16 < 1e-5
