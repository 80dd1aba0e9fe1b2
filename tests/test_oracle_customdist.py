"""Pins of the oracle's customdist (a user-defined two-Gaussian density with
Gaussian observations): the closed form against numerical quadrature, its
special cases, and likelihood weighting against the closed form."""
import numpy as np
import pytest


def _quadrature(prm, y):
    w1, mu1, s1, mu2, s2, r = prm
    x = np.linspace(-25.0, 25.0, 400001)
    prior = (w1 * np.exp(-0.5 * ((x - mu1) / s1) ** 2) / (s1 * np.sqrt(2 * np.pi))
             + (1 - w1) * np.exp(-0.5 * ((x - mu2) / s2) ** 2) / (s2 * np.sqrt(2 * np.pi)))
    loglik = np.zeros_like(x)
    for yj in np.asarray(y, dtype=np.float64):
        loglik += -0.5 * np.log(2 * np.pi * r * r) - (yj - x) ** 2 / (2 * r * r)
    m = loglik.max()
    f = prior * np.exp(loglik - m)
    z = np.trapezoid(f, x)
    mean = np.trapezoid(f * x, x) / z
    var = np.trapezoid(f * (x - mean) ** 2, x) / z
    return m + np.log(z), mean, var


@pytest.mark.parametrize("kw,n,seed", [({}, 8, 1), ({}, 1, 2), (dict(w1=0.8, mu1=3.0, s1=0.2), 20, 3),
                                       (dict(obs_sigma=0.3), 5, 4)])
def test_closed_form_against_quadrature(orc, kw, n, seed):
    prm = orc.customdist_params(**kw)
    y = np.random.default_rng(seed).normal(0.5, 1.5, n).astype(np.float32)
    ex = orc.customdist_exact(prm, y)
    lz, mean, var = _quadrature(prm, y)
    assert ex["log_z"] == pytest.approx(lz, abs=1e-7)
    assert ex["mean"] == pytest.approx(mean, abs=1e-7)
    assert ex["var"] == pytest.approx(var, rel=1e-6)


def test_no_observations_is_the_prior(orc):
    prm = orc.customdist_params()
    ex = orc.customdist_exact(prm, np.zeros(0, np.float32))
    w1, mu1, s1, mu2, s2, _ = prm
    mean = w1 * mu1 + (1 - w1) * mu2
    assert ex["log_z"] == pytest.approx(0.0, abs=1e-15)
    assert ex["mean"] == pytest.approx(mean, rel=1e-12)
    assert ex["var"] == pytest.approx(w1 * (s1 ** 2 + mu1 ** 2) + (1 - w1) * (s2 ** 2 + mu2 ** 2)
                                      - mean ** 2, rel=1e-12)
    x, lw = orc.customdist_is(prm, np.zeros(0, np.float32), 200000, 9)
    assert np.all(lw == 0.0)
    assert x.mean() == pytest.approx(mean, abs=5 * np.sqrt(ex["var"] / 200000))


def test_likelihood_weighting_converges_to_closed_form(orc):
    prm = orc.customdist_params()
    y = np.random.default_rng(7).normal(1.0, 1.0, 6).astype(np.float32)
    ex = orc.customdist_exact(prm, y)
    x, lw = orc.customdist_is(prm, y, 1 << 18, 3)
    m = lw.max()
    w = np.exp(lw - m)
    ess = w.sum() ** 2 / (w ** 2).sum()
    assert m + np.log(w.mean()) == pytest.approx(ex["log_z"], abs=6 / np.sqrt(ess) + 1e-3)
    mean = np.sum(w * x) / w.sum()
    assert mean == pytest.approx(ex["mean"], abs=6 * np.sqrt(ex["var"] / ess))
