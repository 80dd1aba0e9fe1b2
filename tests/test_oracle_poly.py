"""Pins for the oracle's line-fitting traces, normalisation and posterior summary.

The closed form that pins them is the conjugate evidence of Bayesian linear
regression per degree (itself pinned here by numerical quadrature); likelihood
weighting must converge to it where the prior proposal has a large ESS.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

import synth


def test_blr_evidence_matches_quadrature_1d(orc):
    x, y = synth.poly_dataset(5, 11)
    sigma, s = 0.7, 2.0

    def integrand(c0):
        r = y.astype(np.float64) - c0
        return stats.norm.pdf(c0, 0, s) * np.exp(-np.sum(r * r) / (2 * sigma ** 2))

    val, _ = integrate.quad(integrand, -20, 20, epsabs=0, epsrel=1e-12, limit=200)
    lz, mean, var = orc.blr_evidence(x, y, 1, sigma, s)
    assert lz == pytest.approx(math.log(val), abs=1e-9)
    m1, _ = integrate.quad(lambda c: c * integrand(c), -20, 20, epsabs=0, epsrel=1e-12, limit=200)
    assert mean[0] == pytest.approx(m1 / val, rel=1e-8)


def test_blr_evidence_matches_quadrature_2d(orc):
    x, y = synth.poly_dataset(6, 12)
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    sigma, s = 0.8, 1.5

    def integrand(c1, c0):
        r = y64 - c0 - c1 * x64
        return (stats.norm.pdf(c0, 0, s) * stats.norm.pdf(c1, 0, s)
                * np.exp(-np.sum(r * r) / (2 * sigma ** 2)))

    val, _ = integrate.dblquad(integrand, -12, 12, -12, 12, epsabs=0, epsrel=1e-10)
    lz, _, var = orc.blr_evidence(x, y, 2, sigma, s)
    assert lz == pytest.approx(math.log(val), abs=1e-7)
    assert np.all(var > 0)


def test_blr_evidence_no_data_is_zero(orc):
    # with no observations the factor is 1 and the evidence is the prior's mass, 1
    lz, mean, var = orc.blr_evidence(np.zeros(0), np.zeros(0), 3, 0.5, 10.0)
    assert lz == pytest.approx(0.0, abs=1e-12)
    assert np.allclose(mean, 0) and np.allclose(var, 100.0)


def _replicates(orc, model, x, y, N, seeds):
    zs, pns, means = [], [], []
    for s in seeds:
        r, _ = orc.infer_is_poly(model, x, y, N, s)
        zs.append(r["log_z"])
        pns.append(r["p_n"])
        means.append(r["deg_mean"])
    return np.array(zs), np.array(pns), np.array(means)


@pytest.mark.parametrize("L,sigma,prior_sigma,coef_offset", [
    (4, 5.0, 10.0, 1), (8, 2.0, 3.0, 1), (8, 2.0, 3.0, 0)])
def test_is_converges_to_conjugate_evidence(orc, L, sigma, prior_sigma, coef_offset):
    x, y = synth.poly_dataset(L, 21)
    model = orc.poly_model(obs_sigma=sigma, prior_sigma=prior_sigma, coef_offset=coef_offset)
    exact = orc.poly_exact(model, x, y)
    zs, pns, _ = _replicates(orc, model, x, y, 1 << 16, range(8))
    se = zs.std(ddof=1) / math.sqrt(len(zs))
    assert abs(zs.mean() - exact["log_z"]) < 4 * se + 1e-3, (zs.mean(), exact["log_z"], se)
    pn_se = pns.std(axis=0, ddof=1) / math.sqrt(len(zs))
    assert np.all(np.abs(pns.mean(axis=0) - exact["p_n"]) < 4 * pn_se + 2e-3)


def test_is_posterior_moments_converge(orc):
    x, y = synth.poly_dataset(8, 22)
    model = orc.poly_model(obs_sigma=2.0, prior_sigma=3.0)
    exact = orc.poly_exact(model, x, y)
    r, _ = orc.infer_is_poly(model, x, y, 1 << 19, 5)
    for d in range(4):
        nc = 2 + d + 1
        sd = np.sqrt(exact["deg_var"][d, :nc])
        # per-degree ESS is large here; allow 5 posterior sd / sqrt(ESS_d) with ESS_d >= 1000
        assert np.all(np.abs(r["deg_mean"][d, :nc] - exact["deg_mean"][d, :nc]) < 0.16 * sd)
        assert np.all(np.abs(r["deg_var"][d, :nc] / exact["deg_var"][d, :nc] - 1) < 0.25)


def test_prior_draws(orc):
    model = orc.poly_model()
    lw, n, c = orc.is_poly(model, np.zeros(0), np.zeros(0), 40000, 9)
    assert np.all(lw == 0.0)  # no data: every factor is 0
    counts = np.bincount(n - 2, minlength=4)
    assert stats.chisquare(counts).pvalue > 1e-4
    for d in range(2, 6):
        sel = n == d
        assert np.all(c[sel, d + 1:] == 0.0)
        assert stats.kstest(c[sel, :d + 1].ravel() / 10.0, "norm").pvalue > 1e-4


def test_trace_distance_special_cases(orc):
    # tiny prior sd: every coefficient ~0, so lw -> -sum y^2 / (2 sigma^2)
    x, y = synth.poly_dataset(16, 3)
    model = orc.poly_model(prior_sigma=1e-9)
    lw, _, _ = orc.is_poly(model, x, y, 64, 1)
    ref = -np.sum(y.astype(np.float64) ** 2) / (2 * 0.25)
    assert np.allclose(lw, ref, rtol=1e-7)
    # data exactly on a line the trace drew: that trace's distance is 0
    lw1, n1, c1 = orc.poly_trace(orc.poly_model(), np.zeros(0), np.zeros(0), 4, 0, 17)
    xs = np.linspace(-1, 1, 9)
    ys = sum(c1[k] * xs ** k for k in range(n1 + 1))
    lw2, _, _ = orc.poly_trace(orc.poly_model(), xs, ys, 4, 0, 17)
    assert -1e-20 < lw2 <= 0.0


def test_lse_ess_closed_forms(orc):
    N = 1000
    r = orc.lse_ess(np.full(N, -3.5))
    assert r["ess"] == pytest.approx(N, rel=1e-12)
    assert r["lse"] == pytest.approx(-3.5 + math.log(N), abs=1e-12)
    assert r["log_z"] == pytest.approx(-3.5, abs=1e-12)
    onehot = np.full(N, -np.inf)
    onehot[417] = 2.0
    r = orc.lse_ess(onehot)
    assert r["ess"] == 1.0 and r["argmax"] == 417 and r["lse"] == 2.0
    # two levels: k at a, N - k at b
    k, a, b = 37, 0.0, -1.3
    lw = np.full(N, b)
    lw[:k] = a
    r = orc.lse_ess(lw)
    s = k * math.exp(a) + (N - k) * math.exp(b)
    s2 = k * math.exp(2 * a) + (N - k) * math.exp(2 * b)
    assert r["ess"] == pytest.approx(s * s / s2, rel=1e-12)
    assert r["lse"] == pytest.approx(math.log(s), rel=1e-12)
    # against the library routine on a wide random vector
    lw = np.random.default_rng(0).normal(-500, 40, 5000)
    assert orc.lse_ess(lw)["lse"] == pytest.approx(special.logsumexp(lw), abs=1e-9)


def test_lse_argmax_lowest_index_on_ties(orc):
    lw = np.array([-1.0, 4.0, 2.0, 4.0, 4.0])
    assert orc.lse_ess(lw)["argmax"] == 1


def test_posterior_summary_against_library_weighted_stats(orc):
    rng = np.random.default_rng(4)
    N = 5000
    model = orc.poly_model()
    n = rng.integers(2, 6, N).astype(np.int32)
    c = rng.normal(0, 3, (N, 6))
    for i in range(N):
        c[i, n[i] + 1:] = 0
    lw = rng.normal(-20, 2, N)
    r = orc.posterior_poly(model, lw, n, c)
    w = np.exp(lw - lw.max())
    for d in range(4):
        sel = n == d + 2
        assert r["p_n"][d] == pytest.approx(w[sel].sum() / w.sum(), rel=1e-10)
        avg = np.average(c[sel], axis=0, weights=w[sel])
        assert np.allclose(r["deg_mean"][d], avg, rtol=1e-10, atol=1e-12)
        var = np.average((c[sel] - avg) ** 2, axis=0, weights=w[sel])
        assert np.allclose(r["deg_var"][d], var, rtol=1e-9, atol=1e-12)
    assert np.allclose(r["mean_c"], np.average(c, axis=0, weights=w), rtol=1e-10, atol=1e-12)
    assert r["map_deg"] == 2 + int(np.argmax(r["p_n"]))
    assert r["argmax"] == int(np.argmax(lw))
    # equal weights: frequencies and plain sample moments
    r = orc.posterior_poly(model, np.zeros(N), n, c)
    assert np.allclose(r["p_n"], np.bincount(n - 2, minlength=4) / N)
    assert r["ess"] == pytest.approx(N)
