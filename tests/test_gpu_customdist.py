"""customdist (a user-defined two-Gaussian density, observed at every data
point) on the GPU: equal-seed parity with the oracle's likelihood weighting --
draws and log-weights within FP32, the summary within the derived bounds --
and agreement with the closed-form evidence and posterior moments within the
sampling error."""
import numpy as np
import pytest

from gpu_util import load_ppl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppl():
    return load_ppl()


def _run(ppl, orc, kw, y, N, seed):
    import torch
    model = ppl.customdist_model(**{("sigma1" if k == "s1" else "sigma2" if k == "s2" else k): v
                                    for k, v in kw.items()})
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).cuda() if len(y) else None
    x = torch.empty(N, dtype=torch.float32, device="cuda")
    lw = torch.empty(N, dtype=torch.float32, device="cuda")
    res = ppl.ppl_infer_customdist(model, yd, N, seed, x_out=x, lw_out=lw)
    return res, x.cpu().numpy(), lw.cpu().numpy(), orc.customdist_params(**kw)


@pytest.mark.parametrize("kw,n,N", [({}, 8, 100003), (dict(w1=0.8, mu1=3.0, s1=0.2), 20, 65536),
                                    (dict(obs_sigma=0.3), 5, 4097), ({}, 0, 1000), ({}, 5000, 3000)])
def test_customdist_matches_oracle(ppl, orc, kw, n, N):
    y = np.random.default_rng(n).normal(0.5, 1.5, n).astype(np.float32)
    res, x, lw, prm = _run(ppl, orc, kw, y, N, 13)
    xr, lwr = orc.customdist_is(prm, y, N, 13)
    assert res["status"] == 0
    assert np.allclose(x, xr, rtol=1e-5, atol=1e-5)            # same component, FP32 Box-Muller
    assert np.all(np.abs(lw - lwr) <= 4e-6 * np.abs(lwr) + 1e-3)
    m = lwr.max()
    w = np.exp(lwr - m)
    assert res["log_z"] == pytest.approx(m + np.log(w.mean()), abs=1e-3 + 2.0 ** -21 * abs(m))
    assert res["ess"] == pytest.approx(w.sum() ** 2 / (w ** 2).sum(), rel=1e-3)
    mean = np.sum(w * xr) / w.sum()
    var = np.sum(w * (xr - mean) ** 2) / w.sum()
    assert res["mean_x"] == pytest.approx(mean, rel=1e-4, abs=1e-4 * np.sqrt(var))
    assert res["var_x"] == pytest.approx(var, rel=1e-3)


def test_customdist_matches_closed_form(ppl, orc):
    y = np.random.default_rng(3).normal(1.0, 1.0, 6).astype(np.float32)
    res, _, _, prm = _run(ppl, orc, {}, y, 1 << 22, 5)
    ex = orc.customdist_exact(prm, y)
    assert res["log_z"] == pytest.approx(ex["log_z"], abs=6 / np.sqrt(res["ess"]) + 1e-3)
    assert res["mean_x"] == pytest.approx(ex["mean"], abs=6 * np.sqrt(ex["var"] / res["ess"]))
    assert res["var_x"] == pytest.approx(ex["var"], rel=0.05)
