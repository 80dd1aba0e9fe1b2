"""Pins for exact enumeration and for likelihood weighting on tiny discrete models.

Enumeration is checked against closed forms (Bayes' rule on a grid prior, the
binomial pmf from scipy, the truncated geometric pmf); likelihood weighting is
checked to converge to the enumerated posterior within binomial error.
"""
import numpy as np
import pytest
from scipy import stats

FLIPS = [1, 1, 0, 1, 1, 1, 0, 1]


def test_biasedcoin_enumeration_is_bayes_rule(orc):
    vals, probs = orc.enumerate_model("biasedcoin", FLIPS)
    theta = np.arange(1, 10) / 10
    h = sum(FLIPS)
    lik = theta ** h * (1 - theta) ** (len(FLIPS) - h)
    assert np.allclose(vals, theta)
    assert np.allclose(probs, lik / lik.sum(), rtol=1e-12)


def test_binomial_enumeration_is_binomial_pmf(orc):
    vals, probs = orc.enumerate_model("binomial", [7])
    assert np.allclose(vals, np.arange(8))
    assert np.allclose(probs, stats.binom.pmf(np.arange(8), 7, 0.3), rtol=1e-12)


def test_geometric_enumeration_truncated(orc):
    vals, probs = orc.enumerate_model("geometric", [12])
    c = np.arange(12)
    ref = 0.5 ** (c + 1)
    assert np.allclose(vals, c) and np.allclose(probs, ref / ref.sum(), rtol=1e-12)
    vals, _ = orc.enumerate_model("geometric", [12], max_depth=5)
    assert len(vals) == 5


@pytest.mark.parametrize("name,data", [("biasedcoin", FLIPS), ("binomial", [6]),
                                       ("geometric", [8])])
def test_likelihood_weighting_converges_to_enumeration(orc, name, data):
    vals, probs = orc.enumerate_model(name, data)
    N = 200000
    v, lw = orc.is_discrete(name, data, N, 31)
    w = np.exp(lw - lw[np.isfinite(lw)].max())
    w[~np.isfinite(lw)] = 0
    W = w / w.sum()
    ess = 1 / np.sum(W ** 2)
    for val, p in zip(vals, probs):
        est = W[v == val].sum()
        assert abs(est - p) < 5 * np.sqrt(p * (1 - p) / ess) + 1e-4, (val, est, p)
