"""Likelihood weighting on the paper's tiny discrete benchmarks (biasedcoin,
binomial, truncated geometric) against the oracle at equal seeds -- return
values and per-value counts bit-exact, log-weights within FP32, the
normalised distribution within FP64 rounding -- and against exact
enumeration within the sampling error."""
import math

import numpy as np
import pytest

from gpu_util import load_ppl

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(12)
FLIPS_SHORT = [1, 1, 0, 1, 0, 1, 1, 1, 0, 1]
FLIPS_LONG = list((RNG.random(200) < 0.7).astype(int))
CASES = [("biasedcoin", FLIPS_SHORT, 0), ("biasedcoin", FLIPS_LONG, 0), ("biasedcoin", [], 0),
         ("binomial", None, 10), ("binomial", None, 0), ("binomial", None, 63),
         ("geometric", None, 12), ("geometric", None, 1)]


@pytest.fixture(scope="module")
def ppl():
    return load_ppl()


def _run(ppl, name, N, seed, flips, limit):
    import torch
    codes = torch.empty(N, dtype=torch.int32, device="cuda")
    lw = torch.empty(N, dtype=torch.float32, device="cuda")
    fl = None if not flips else torch.tensor(flips, dtype=torch.int32, device="cuda")
    res = ppl.ppl_infer_discrete(name, N, seed, flips=fl, limit=limit, codes_out=codes, lw_out=lw)
    return res, codes.cpu().numpy(), lw.cpu().numpy()


def _oracle_data(name, flips, limit):
    return np.array(flips, dtype=np.int32) if name == "biasedcoin" else np.array([limit], np.int32)


@pytest.mark.parametrize("name,flips,limit", CASES)
def test_discrete_matches_oracle(ppl, orc, name, flips, limit):
    N = 100003
    res, codes, lw = _run(ppl, name, N, 21, flips, limit)
    vals, lw_r = orc.is_discrete(name, _oracle_data(name, flips, limit), N, 21)
    got = (codes + 1) / 10.0 if name == "biasedcoin" else codes.astype(np.float64)
    assert np.array_equal(np.round(got * 10), np.round(vals * 10))   # return values: exact
    fin = np.isfinite(lw_r)
    assert np.array_equal(np.isfinite(lw), fin)
    assert np.allclose(lw[fin], lw_r[fin], rtol=1e-5, atol=1e-5)
    n_values = 9 if name == "biasedcoin" else limit + 1
    assert res["status"] == 0 and res["n_values"] == n_values
    assert np.array_equal(res["count"], np.bincount(codes, minlength=n_values))
    # the oracle's normalised distribution, in FP64 from its own values and weights
    m = lw_r[fin].max()
    w = np.where(fin, np.exp(np.where(fin, lw_r, 0.0) - m), 0.0)
    prob = np.bincount(codes, weights=w, minlength=n_values) / w.sum()
    assert np.allclose(res["prob"], prob, rtol=1e-12, atol=1e-15)
    assert res["log_z"] == pytest.approx(m + np.log(w.sum()) - np.log(N), rel=1e-12, abs=1e-12)
    assert res["ess"] == pytest.approx(w.sum() ** 2 / (w ** 2).sum(), rel=1e-10)


@pytest.mark.parametrize("name,flips,limit", CASES)
def test_discrete_matches_enumeration(ppl, orc, name, flips, limit):
    N = 1 << 20
    res, _, _ = _run(ppl, name, N, 5, flips, limit)
    exact = np.zeros(res["n_values"])
    if name == "binomial" and limit > 20:  # beyond enumeration: the binomial pmf
        for k in range(limit + 1):
            exact[k] = math.comb(limit, k) * 0.3 ** k * 0.7 ** (limit - k)
    else:
        vals, probs = orc.enumerate_model(name, _oracle_data(name, flips, limit))
        for v, p in zip(vals, probs):
            exact[int(round(v * 10)) - 1 if name == "biasedcoin" else int(v)] = p
    # sampling error of self-normalised weights: sd <= sqrt(p (1 - p) / ESS)
    sd = np.sqrt(exact * (1 - exact) / res["ess"])
    assert np.all(np.abs(res["prob"] - exact) <= 6 * sd + 1e-9), (res["prob"], exact)
    mean = float(np.sum(exact * res["value"]))
    spread = np.sqrt(np.sum(exact * (res["value"] - mean) ** 2) / res["ess"])
    assert abs(res["mean"] - mean) <= 6 * spread + 1e-9
