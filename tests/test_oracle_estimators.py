"""Pins for the oracle's classical estimator (Section 3) and the learned
Beta prior (Section 4.1)."""
import math

import numpy as np
import pytest

import oracle as O
import synth


@pytest.mark.parametrize("kind,n", [(O.JACCARD, 360), (O.COSINE, 2048)])
def test_mle_unbiased_with_binomial_variance(kind, n):
    """Section 3: m/n is unbiased for the agreement probability with variance
    s(1-s)/n; for cosine the estimate of the angle is pi (1 - m/n)."""
    s = 0.8
    P = 4000
    sig, pairs = synth.bernoulli_signatures(np.full(P, s), n, "jaccard" if kind == O.JACCARD else "cosine", seed=2)
    m, est, keep = O.estimate_mle(kind, n, 0.7, pairs, sig)
    r = m.astype(np.float64) / n
    assert abs(r.mean() - s) < 4 * math.sqrt(s * (1 - s) / n / P)
    assert r.var() == pytest.approx(s * (1 - s) / n, rel=0.1)
    if kind == O.COSINE:
        assert np.allclose(np.arccos(np.clip(est, -1, 1)), math.pi * (1 - r), atol=1e-12)
    else:
        assert np.array_equal(est, r)
    assert np.array_equal(keep, (est > 0.7).astype(np.uint8))


def test_mle_agreement_counts_brute_force():
    sig, pairs = synth.bernoulli_signatures(np.array([0.3, 0.9, 1.0, 0.0]), 96, "cosine", seed=4)
    m, _, _ = O.estimate_mle(O.COSINE, 70, 0.5, pairs, sig)   # a partial last word
    bits = np.unpackbits(sig.view(np.uint8), axis=1, bitorder="little")[:, :70]
    assert m.tolist() == [int((bits[2 * i] == bits[2 * i + 1]).sum()) for i in range(4)]


def test_prior_hand_example():
    """mean 0.4, variance (0.04 + 0 + 0.04)/3, so s(1-s)/v - 1 = 8:
    alpha = 3.2, beta = 4.8."""
    mean, var, a, b, fb = O.fit_beta_prior(np.array([0.2, 0.4, 0.6]))
    assert mean == pytest.approx(0.4) and var == pytest.approx(0.08 / 3)
    assert (a, b, fb) == (pytest.approx(3.2), pytest.approx(4.8), 0.0)


def test_prior_recovers_beta_parameters():
    rng = np.random.default_rng(1)
    for a0, b0 in ((2.0, 5.0), (0.7, 0.9), (8.0, 3.0)):
        _, _, a, b, fb = O.fit_beta_prior(rng.beta(a0, b0, 400000))
        assert fb == 0.0 and a == pytest.approx(a0, rel=0.03) and b == pytest.approx(b0, rel=0.03)


def test_prior_fallback_when_no_beta_fits():
    assert O.fit_beta_prior(np.full(10, 0.25))[2:] == (1.0, 1.0, 1.0)        # zero variance
    assert O.fit_beta_prior(np.array([0.0, 1.0]))[2:] == (1.0, 1.0, 1.0)     # v = s(1-s)
