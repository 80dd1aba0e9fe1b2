"""Pins for the oracle's state-space model: Kalman filter and SMC.

The Kalman log-evidence is pinned by the dense joint-Gaussian density of the
observations (scipy's multivariate normal); the SMC estimate by the Kalman
value, statistically over seeds.
"""
import math

import numpy as np
import pytest
from scipy import stats

import synth


def _joint_logpdf(y, phi, q, r):
    T = len(y)
    cov = np.zeros((T, T))
    for t in range(T):
        for s in range(T):
            # x_t = sum_{k<=t} phi^(t-k) q e_k (x_0 = 0, steps 1..t)
            cov[t, s] = sum(phi ** (t - k) * phi ** (s - k) * q * q for k in range(min(t, s) + 1))
    cov += r * r * np.eye(T)
    return stats.multivariate_normal(mean=np.zeros(T), cov=cov).logpdf(y)


@pytest.mark.parametrize("T,phi,q,r", [(1, 0.9, 1.0, 0.5), (5, 0.9, 1.0, 0.5),
                                       (10, -0.5, 0.3, 2.0), (8, 1.0, 1.0, 1.0)])
def test_kalman_matches_joint_gaussian(orc, T, phi, q, r):
    y = synth.lgssm_dataset(T, 7, phi, q, r).astype(np.float64)
    lz = orc.kalman_logz(orc.lgssm_model(phi, q, r), y)
    assert lz == pytest.approx(_joint_logpdf(y, phi, q, r), abs=1e-10)


@pytest.mark.parametrize("state_f32", [False, True])
def test_smc_converges_to_kalman(orc, state_f32):
    model = orc.lgssm_model()
    y = synth.lgssm_dataset(50, 2)
    exact = orc.kalman_logz(model, y)
    zs = np.array([orc.smc_lgssm(model, y, 1 << 12, s, state_f32)["log_z"] for s in range(16)])
    se = zs.std(ddof=1) / math.sqrt(len(zs))
    # SMC's evidence estimate is unbiased in Z, so log Z is biased low by ~var/2
    bias = zs.var(ddof=1) / 2
    assert abs(zs.mean() + bias - exact) < 4 * se + 1e-3, (zs.mean(), exact, se)


def test_smc_resampling_rule(orc):
    model = orc.lgssm_model()
    y = synth.lgssm_dataset(30, 4)
    out = orc.smc_lgssm(model, y, 2000, 1)
    N = 2000
    assert np.array_equal(out["resampled"], (out["ess"] < N / 2).astype(np.int32))
    assert out["resampled"].sum() > 0
    if out["resampled"][-1]:
        assert np.all(out["lw"] == 0)


def test_smc_single_particle_is_prior_path(orc):
    # with N = 1 every step resamples nothing new: ESS = 1 >= 1/2, so no resampling,
    # and log Z is the sum of the observe terms along the one prior path
    model = orc.lgssm_model()
    y = synth.lgssm_dataset(6, 5)
    out = orc.smc_lgssm(model, y, 1, 3)
    assert out["resampled"].sum() == 0
    assert out["log_z"] == pytest.approx(out["lw"][0], abs=1e-12)


def test_smc_fp32_state_is_rounded_fp64_state(orc):
    # one step without resampling: the FP32 state is the FP64 update in FP32 rounding
    model = orc.lgssm_model()
    y = synth.lgssm_dataset(1, 3)
    a = orc.smc_lgssm(model, y, 64, 5, False)
    b = orc.smc_lgssm(model, y, 64, 5, True)
    assert np.allclose(a["x"], b["x"], rtol=3e-7, atol=1e-7)
    assert np.allclose(a["lw"], b["lw"], rtol=1e-6, atol=1e-6)
    assert np.all(b["x"] == b["x"].astype(np.float32))
