"""Pins for the oracle of the learned proposal: BF16 rounding and the network
against torch's library routines, log q against scipy, the gradient against
central finite differences, and importance sampling under a learned proposal
against the prior special case and the conjugate closed form."""
import math

import numpy as np
import pytest
from scipy import special, stats

import synth


@pytest.fixture(scope="module")
def mlp(orc):
    from oracle import mlp
    return mlp


def test_bf16_rounding_matches_torch(mlp):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(0, 10, 3000), rng.normal(0, 1e-3, 1000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.0078125, 65504.0]]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([mlp.bf16(x) for x in v], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_features_sorted_and_rounded(mlp):
    torch = pytest.importorskip("torch")
    x, y = synth.poly_dataset(32, 5)
    f = mlp.features(x, y)
    order = np.argsort(x, kind="stable")
    ref = np.empty(64, dtype=np.float32)
    ref[0::2] = x[order]
    ref[1::2] = y[order] / np.float32(10.0)
    ref = torch.from_numpy(ref).to(torch.bfloat16).float().numpy()
    assert np.array_equal(f, ref)


def test_forward_matches_torch_linear(mlp):
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    W = synth.mlp_weights(3)
    x, y = synth.poly_dataset(32, 9)
    feat = mlp.features(x, y)
    out, h1, h2 = mlp.forward(W, feat)
    t = [torch.from_numpy(w).double() for w in W]
    r = lambda v: v.float().to(torch.bfloat16).double()
    a1 = r(F.relu(F.linear(torch.from_numpy(feat).double(), t[0], t[1])))
    a2 = r(F.relu(F.linear(a1, t[2], t[3])))
    o = F.linear(a2, t[4], t[5])
    assert np.allclose(h1, a1.numpy(), rtol=0, atol=0) or np.mean(h1 != a1.numpy()) < 0.01
    assert np.allclose(out, o.numpy(), rtol=1e-6, atol=1e-6)


def test_proposal_logq_matches_scipy(mlp, orc):
    m = orc.poly_model()
    rng = np.random.default_rng(2)
    out = rng.normal(0, 1, 48)
    for n in range(2, 6):
        k = n - 2
        c = rng.normal(0, 10, 6)
        lq, _ = mlp.proposal_logq(m, out, n, c)
        base = sum(2 + kk + 1 for kk in range(k))
        ref = special.log_softmax(out[:4])[k]
        for j in range(n + 1):
            mu = 10 * out[4 + 2 * (base + j)]
            t = np.clip(out[5 + 2 * (base + j)], -9, 1)
            ref += stats.norm.logpdf(c[j], mu, 10 * np.exp(t))
        assert lq == pytest.approx(ref, rel=1e-12)


def test_loss_gradient_matches_finite_differences(mlp, orc):
    m = orc.poly_model()
    W = synth.mlp_weights(4, bias_scale=0.5)
    pairs = [mlp.forward_sim(m, 11, p) for p in range(6)]
    feats = np.stack([mlp.features(x, y) for x, y, _, _ in pairs])
    n = np.array([p[2] for p in pairs])
    c = np.stack([p[3] for p in pairs])
    mlp.set_bf16(False)
    try:
        loss, g = mlp.loss_grad(m, W, feats, n, c)
        rng = np.random.default_rng(5)
        for wi in range(6):
            flat = W[wi].reshape(-1)
            for idx in rng.choice(flat.size, 6, replace=False):
                eps = np.float32(1e-2) * max(1.0, abs(flat[idx]))
                Wp = [w.copy() for w in W]
                Wm = [w.copy() for w in W]
                Wp[wi].reshape(-1)[idx] += eps
                Wm[wi].reshape(-1)[idx] -= eps
                dp = float(Wp[wi].reshape(-1)[idx]) - float(W[wi].reshape(-1)[idx])
                dm = float(W[wi].reshape(-1)[idx]) - float(Wm[wi].reshape(-1)[idx])
                lp, _ = mlp.loss_grad(m, Wp, feats, n, c, with_grad=False)
                lm, _ = mlp.loss_grad(m, Wm, feats, n, c, with_grad=False)
                fd = (lp - lm) / (dp + dm)
                an = g[wi].reshape(-1)[idx]
                assert abs(fd - an) <= 2e-3 * max(1.0, abs(an)) + 1e-4 * abs(loss), (wi, idx, fd, an)
    finally:
        mlp.set_bf16(True)


def test_prior_equal_proposal_reproduces_prior_traces(mlp, orc):
    m = orc.poly_model()
    out = np.zeros(48)  # uniform degree logits, mu = 0, s = prior_sigma
    x, y = synth.poly_dataset(32, 0)
    lw, n, c = mlp.learned_is(m, out, x, y, 4000, 3)
    lw0, n0, c0 = orc.is_poly(m, x, y, 4000, 3)
    assert np.array_equal(n, n0) and np.array_equal(c, c0) and np.array_equal(lw, lw0)


def _conjugate_proposal(orc, x, y, temper=1.0):
    m = orc.poly_model()
    ex = orc.poly_exact(m, x, y)
    out = np.zeros(48)
    out[:4] = np.log(ex["p_n"] + 1e-300)
    base = 0
    for k in range(4):
        nc = 3 + k
        for j in range(nc):
            out[4 + 2 * (base + j)] = ex["deg_mean"][k, j] / 10.0
            out[5 + 2 * (base + j)] = np.log(temper * np.sqrt(ex["deg_var"][k, j]) / 10.0)
        base += nc
    return out, ex


def test_good_proposal_gives_the_exact_evidence(mlp, orc):
    # a proposal close to the posterior (the conjugate marginals, widened) has a
    # large ESS, and importance weighting recovers the closed-form evidence
    x, y = synth.poly_dataset(32, 0)
    out, ex = _conjugate_proposal(orc, x, y, temper=1.5)
    m = orc.poly_model()
    zs, esss = [], []
    for s in range(6):
        lw, _, _ = mlp.learned_is(m, out, x, y, 1 << 15, s)
        r = orc.lse_ess(lw)
        zs.append(r["log_z"])
        esss.append(r["ess"])
    zs = np.array(zs)
    assert min(esss) > 1000
    se = zs.std(ddof=1) / math.sqrt(len(zs))
    assert abs(zs.mean() - ex["log_z"]) < 4 * se + 0.01


def test_any_proposal_is_unbiased(mlp, orc):
    # a poor but valid proposal still targets the same evidence (Z estimates unbiased)
    x, y = synth.poly_dataset(6, 4)
    m = orc.poly_model(obs_sigma=3.0, prior_sigma=3.0)
    ex = orc.poly_exact(m, x, y)
    rng = np.random.default_rng(8)
    out = rng.normal(0, 0.3, 48)
    zs = np.array([orc.lse_ess(mlp.learned_is(m, out, x, y, 1 << 14, s)[0])["log_z"]
                   for s in range(10)])
    se = zs.std(ddof=1) / math.sqrt(len(zs))
    assert abs(zs.mean() + zs.var(ddof=1) / 2 - ex["log_z"]) < 4 * se + 0.01


def test_forward_simulation_distribution(mlp, orc):
    m = orc.poly_model()
    pairs = [mlp.forward_sim(m, 21, p) for p in range(3000)]
    n = np.array([p[2] for p in pairs])
    assert stats.chisquare(np.bincount(n - 2, minlength=4)).pvalue > 1e-4
    xs = np.concatenate([p[0] for p in pairs])
    assert stats.kstest((xs + 1) / 2, "uniform").pvalue > 1e-4
    res = []
    for x, y, nn, c in pairs:
        f = sum(c[j] * x.astype(np.float64) ** j for j in range(nn + 1))
        res.append((y - f) / 0.5)
    assert stats.kstest(np.concatenate(res), "norm").pvalue > 1e-4
    c0 = np.array([p[3][0] for p in pairs]) / 10.0
    assert stats.kstest(c0, "norm").pvalue > 1e-4
