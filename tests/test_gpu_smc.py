"""Parity of the CUDA bootstrap particle filter with the oracle at equal seeds,
and of its evidence estimate with the Kalman filter.

Resampling turns rounding differences into different ancestors, which then
decorrelate the two runs, so equal-seed parity compares against the oracle's
filter with FP32 state and log-weights (the method's precision policy); the
FP64 filter and the GPU agree with the Kalman evidence statistically."""
import math

import numpy as np
import pytest

import synth
from gpu_util import load_ppl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppl():
    return load_ppl()


def run_smc(ppl, y, N, seed):
    import torch
    model = ppl.lgssm_model()
    x = torch.zeros(N, dtype=torch.float32, device="cuda")
    lw = torch.zeros(N, dtype=torch.float32, device="cuda")
    acc = torch.zeros(1, dtype=torch.float64, device="cuda")
    flags = torch.zeros(len(y), dtype=torch.int32, device="cuda")
    est = torch.zeros((len(y), 2), dtype=torch.float64, device="cuda")
    ws = ppl.workspace(model, N)
    for t in range(1, len(y) + 1):
        ppl.ppl_smc_step(model, float(y[t - 1]), t, seed, x, lw, acc, flags[t - 1:t],
                         est[t - 1], ws)
    assert ppl.ppl_workspace_status(ws) == 0
    return {"log_z": float(est[-1, 0]), "ess": est[:, 1].cpu().numpy(),
            "resampled": flags.cpu().numpy(), "x": x.cpu().numpy(), "lw": lw.cpu().numpy()}


@pytest.mark.parametrize("N,T", [(1, 5), (4099, 40), (65536, 100)])
def test_smc_matches_oracle(ppl, orc, N, T):
    y = synth.lgssm_dataset(T, 2)
    g = run_smc(ppl, y, N, 7)
    r = orc.smc_lgssm(orc.lgssm_model(), y, N, 7, state_f32=True)
    assert abs(g["log_z"] - r["log_z"]) <= 1e-3
    # the resampling decisions agree except where the ESS sits on N/2
    diff = g["resampled"] != r["resampled"]
    assert np.all(np.abs(r["ess"][diff] / N - 0.5) < 1e-4)


def test_smc_full_size_matches_oracle_and_kalman(ppl, orc):
    y = synth.lgssm_dataset(200, 2)
    N = 1 << 20
    g = run_smc(ppl, y, N, 2)
    r = orc.smc_lgssm(orc.lgssm_model(), y, N, 2, state_f32=True)
    assert abs(g["log_z"] - r["log_z"]) <= 1e-3
    kal = orc.kalman_logz(orc.lgssm_model(), y)
    assert abs(g["log_z"] - kal) < 0.05


def test_smc_estimates_kalman_evidence(ppl, orc):
    y = synth.lgssm_dataset(200, 2)
    kal = orc.kalman_logz(orc.lgssm_model(), y)
    zs = np.array([run_smc(ppl, y, 1 << 14, s)["log_z"] for s in range(12)])
    se = zs.std(ddof=1) / math.sqrt(len(zs))
    assert abs(zs.mean() + zs.var(ddof=1) / 2 - kal) < 4 * se + 1e-3


def test_first_step_state_is_the_reproducible_normal_bit_for_bit(ppl, orc):
    # after step 1 from x = 0 with phi = 0.9, q = 1: x = 0.9 * 0 + 1 * z = z exactly
    import torch
    N = 100003
    model = ppl.lgssm_model()
    x = torch.zeros(N, dtype=torch.float32, device="cuda")
    lw = torch.zeros(N, dtype=torch.float32, device="cuda")
    acc = torch.zeros(1, dtype=torch.float64, device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    est = torch.zeros(2, dtype=torch.float64, device="cuda")
    ws = ppl.workspace(model, N)
    ppl.ppl_smc_step(model, 0.3, 1, 5, x, lw, acc, flag, est, ws)
    xs = x.cpu().numpy()
    words = ppl.ppl_rng_words(5, 0, 1, 2, N, 1).cpu().numpy().view(np.uint32)
    for i in list(range(0, N, 997)) + [N - 1]:
        ref = np.float32(orc.normal32(int(words[i, 0, 0]), int(words[i, 0, 1])))
        assert xs[i] == ref, (i, xs[i], ref)


@pytest.mark.parametrize("N,T", [(1, 5), (4099, 40), (1 << 20, 200)])
def test_persistent_filter_matches_stepwise_and_oracle(ppl, orc, N, T):
    import torch
    y = synth.lgssm_dataset(T, 2)
    out = ppl.ppl_smc_run(ppl.lgssm_model(), torch.from_numpy(y).cuda(), N, 7)
    assert ppl.ppl_workspace_status(out["ws"]) == 0
    g = run_smc(ppl, y, N, 7)
    assert np.array_equal(out["resampled"].cpu().numpy(), g["resampled"])
    assert np.array_equal(out["x"].cpu().numpy(), g["x"])  # same particles, bit for bit
    assert np.array_equal(out["lw"].cpu().numpy(), g["lw"])
    # the two sum the FP32 block partials in different groupings: ~1e-7 per step
    np.testing.assert_allclose(out["ess"].cpu().numpy(), g["ess"], rtol=1e-5)
    assert abs(float(out["log_z"].item()) - g["log_z"]) < 1e-6 * T
    r = orc.smc_lgssm(orc.lgssm_model(), y, N, 7, state_f32=True)
    assert abs(float(out["log_z"].item()) - r["log_z"]) <= 1e-3


def test_grid_barrier_probe_passes_its_barriers_and_checks_sizes(ppl):
    """The probe behind the bench's barrier floor: the filter's launch shape
    (one 1024-thread block per SM) passes its barriers with a clean status;
    more blocks than SMs, or no barrier, is refused before any launch."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ws = ppl.ppl_grid_barrier_probe(sms, 200)
    torch.cuda.synchronize()
    assert ppl.ppl_workspace_status(ws) == 0
    for blocks, n in ((sms + 1, 10), (1, 0), (0, 10)):
        with pytest.raises(ppl.PplError) as err:
            ppl.ppl_grid_barrier_probe(blocks, n, ws=ws)
        assert err.value.status == ppl.PPL_EINVAL
