"""Parity of the CUDA normalisation, resampling and gather with the oracle.

Ancestors are compared bit for bit: from identical fixed-point weights, and
from identical FP32 log-weights (the FP32 exponential that decides the
integer weights is part of the definition on both sides).
"""
import numpy as np
import pytest

import synth
from gpu_util import load_ppl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppl():
    return load_ppl()


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("N,M", [(1, 1), (2, 5), (2047, 2049), (2048, 2048), (2049, 100),
                                 (100003, 77777), (65536, 300000), (3, 1 << 20),
                                 (40000, 1 << 21)])
def test_fixed_point_ancestors_bit_exact(ppl, orc, N, M):
    q = synth.fixed_weights(N, N + M)
    if q.sum() == 0:
        q[0] = 3
    anc = ppl.ppl_resample(M, 5, instance=2, t=9, q_fixed=_t(q.view(np.int64))).cpu().numpy()
    st, ref = orc.resample_systematic(q, M, 5, 2, 9)
    assert st == 0 and np.array_equal(anc, ref)


@pytest.mark.parametrize("kind", ["normal", "equal", "onehot", "sparse", "wide"])
@pytest.mark.parametrize("N", [1, 777, 4099, 262147])
def test_log_weight_ancestors_bit_exact(ppl, orc, kind, N):
    lw = synth.log_weights(N, 3 + N, kind)
    anc = ppl.ppl_resample(N, 11, t=4, lw=_t(lw)).cpu().numpy()
    st, ref = orc.resample_from_lw(lw, N, 11, 0, 4)
    assert st == 0 and np.array_equal(anc, ref)


@pytest.mark.parametrize("kind", ["normal", "onehot"])
def test_full_size_2_24(ppl, orc, kind):
    N = 1 << 24
    lw = synth.log_weights(N, 12, kind, scale=30.0)
    anc = ppl.ppl_resample(N, 1, t=0, lw=_t(lw)).cpu().numpy()
    st, ref = orc.resample_from_lw(lw, N, 1, 0, 0)
    assert st == 0 and np.array_equal(anc, ref)


def test_gather_records(ppl, orc):
    rng = np.random.default_rng(2)
    for rec_shape, dtype in [((5000, 8), np.float32), ((3001,), np.float32),
                             ((1234, 3), np.int16)]:
        rec = rng.integers(-1000, 1000, rec_shape).astype(dtype)
        anc = np.sort(rng.integers(0, rec_shape[0], 4321)).astype(np.int32)
        out = ppl.ppl_gather(_t(rec), _t(anc)).cpu().numpy()
        assert np.array_equal(out, orc.gather(rec, anc))
    # an ancestor out of range gives a zero record, never a stray read
    rec = np.arange(40, dtype=np.float32).reshape(5, 8)
    out = ppl.ppl_gather(_t(rec), _t(np.array([0, 7, -1, 4], dtype=np.int32))).cpu().numpy()
    assert np.array_equal(out[0], rec[0]) and np.array_equal(out[3], rec[4])
    assert np.all(out[1] == 0) and np.all(out[2] == 0)


@pytest.mark.parametrize("N", [1, 100, 100003, 1 << 24])
def test_logsumexp(ppl, orc, N):
    lw = synth.log_weights(N, 4, "normal", scale=20.0)
    out = ppl.ppl_logsumexp(_t(lw)).cpu().numpy()
    ref = orc.lse_ess(lw.astype(np.float64))
    assert out[0] == pytest.approx(ref["lse"], abs=1e-5)
    assert out[1] == pytest.approx(ref["ess"], rel=1e-5)
    assert out[2] == ref["max_lw"] and int(out[3]) == ref["argmax"]


@pytest.mark.parametrize("N", [16, 100003, 1 << 20])
def test_logsumexp_ties_and_misaligned_input(ppl, orc, N):
    # the maximum at several indices: the lowest wins, in the vector path and in
    # the scalar path a misaligned view takes (offset by one float)
    lw = synth.log_weights(N + 1, 9, "normal", scale=3.0)
    peak = float(lw.max()) + 1.0
    for j in (N // 3, N // 2, N - 1):
        lw[j + 1] = peak
    dev = _t(lw)
    for t, view in ((dev[1:], lw[1:]), (dev[:N], lw[:N])):  # 4 bytes off 16-byte alignment, aligned
        out = ppl.ppl_logsumexp(t).cpu().numpy()
        ref = orc.lse_ess(view.astype(np.float64))
        assert out[0] == pytest.approx(ref["lse"], abs=1e-5)
        assert out[1] == pytest.approx(ref["ess"], rel=1e-5)
        assert out[2] == ref["max_lw"] and int(out[3]) == ref["argmax"]
    const = _t(np.zeros(N, dtype=np.float32))
    out = ppl.ppl_logsumexp(const).cpu().numpy()
    assert int(out[3]) == 0 and out[1] == pytest.approx(N, rel=1e-6)


def test_device_errors_are_reported(ppl):
    import torch
    lw = np.zeros(5000, dtype=np.float32)
    lw[1234] = np.nan
    ws = ppl.workspace(ppl.poly_model(), 5000)
    ppl.ppl_logsumexp(_t(lw), ws=ws)
    assert ppl.ppl_workspace_status(ws) == ppl.PPL_ENAN
    ppl.ppl_logsumexp(_t(np.full(5000, -np.inf, dtype=np.float32)), ws=ws)
    assert ppl.ppl_workspace_status(ws) == ppl.PPL_EEMPTY
    ppl.ppl_resample(5000, 0, q_fixed=_t(np.full(5000, 1 << 60, dtype=np.int64)), ws=ws)
    assert ppl.ppl_workspace_status(ws) == ppl.PPL_EINVAL
    ppl.ppl_resample(5000, 0, q_fixed=_t(np.zeros(5000, dtype=np.int64)), ws=ws)
    assert ppl.ppl_workspace_status(ws) == ppl.PPL_EEMPTY
    ppl.ppl_resample(5000, 0, lw=_t(np.zeros(5000, dtype=np.float32)), ws=ws)
    assert ppl.ppl_workspace_status(ws) == ppl.PPL_OK
    torch.cuda.synchronize()


@pytest.mark.parametrize("kind", ["normal", "onehot", "sparse"])
@pytest.mark.parametrize("N,M", [(1, 1), (4099, 4099), (100003, 100780), (262147, 70001)])
@pytest.mark.parametrize("rec", ["f32x8", "f32x12", "i16x8", "f32x3", "f32x1", "i16x3"])
def test_resample_gather_bit_exact(ppl, orc, kind, N, M, rec):
    # 32-, 48- and 16-byte records take the fused path in 16-byte words, 12-
    # and 4-byte ones in 4-byte words, 6-byte ones the separate gather;
    # ancestors and records against the oracle, bit for bit
    import torch
    rng = np.random.default_rng(N + M)
    cols, dtype = {"f32x8": (8, np.float32), "f32x12": (12, np.float32),
                   "i16x8": (8, np.int16), "f32x3": (3, np.float32), "f32x1": (1, np.float32),
                   "i16x3": (3, np.int16)}[rec]
    state = rng.integers(-30000, 30000, (N, cols)).astype(dtype)
    lw = synth.log_weights(N, 7 + N, kind)
    st, anc_ref = orc.resample_from_lw(lw, M, 13, 1, 3)
    assert st == 0
    for known in (False, True):
        mx = torch.tensor([float(lw.max())], dtype=torch.float64, device="cuda") if known else None
        anc, out = ppl.ppl_resample_gather(M, 13, _t(lw), _t(state), max_lw_dev=mx, instance=1,
                                           t=3)
        assert np.array_equal(anc.cpu().numpy(), anc_ref)
        assert np.array_equal(out.cpu().numpy(), orc.gather(state, anc_ref))


def test_known_max_below_a_log_weight_is_reported(ppl):
    import torch
    lw = synth.log_weights(10000, 5, "normal")
    ws = ppl.workspace(ppl.poly_model(), 10000)
    mx = torch.tensor([float(lw.max()) - 1.0], dtype=torch.float64, device="cuda")
    ppl.ppl_resample_known_max(10000, 1, _t(lw), mx, ws=ws)
    assert ppl.ppl_workspace_status(ws) == ppl.PPL_EINVAL
    mx = torch.tensor([float(lw.max())], dtype=torch.float64, device="cuda")
    ppl.ppl_resample_known_max(10000, 1, _t(lw), mx, ws=ws)
    assert ppl.ppl_workspace_status(ws) == ppl.PPL_OK


def test_known_max_matches_plain_resample(ppl, orc):
    import torch
    x, y = synth.poly_dataset(64, 2)
    N = 300007
    model = ppl.poly_model()
    lw = torch.empty(N, dtype=torch.float32, device="cuda")
    res = ppl.ppl_infer_is(model, _t(x), _t(y), N, 4, lw_out=lw)
    a = ppl.ppl_resample_known_max(N, 3, lw, ppl.result_max_lw(res), t=2)
    b = ppl.ppl_resample(N, 3, t=2, lw=lw)
    assert torch.equal(a, b)
    st, ref = orc.resample_from_lw(lw.cpu().numpy(), N, 3, 0, 2)
    assert st == 0 and np.array_equal(a.cpu().numpy(), ref)


def test_bounded_wait_reports_timeout_and_recovers(ppl):
    # a tile that never publishes makes every later tile's bounded wait expire;
    # the status comes back as PPL_ETIMEOUT and the context stays usable
    import torch
    q = _t(synth.fixed_weights(5 * 2048 + 17, 3).view(np.int64))
    assert ppl.ppl_selftest_scan_timeout(q, 1 << 12) == ppl.PPL_ETIMEOUT
    anc = ppl.ppl_resample(1000, 1, q_fixed=q)
    ws = ppl.workspace(ppl.poly_model(), q.numel())
    ppl.ppl_resample(1000, 1, q_fixed=q, ancestors=anc, ws=ws)
    assert ppl.ppl_workspace_status(ws) == ppl.PPL_OK
    torch.cuda.synchronize()


@pytest.mark.parametrize("source", ["linefitting", "normal"])
def test_resample_gather_full_size_2_24(ppl, orc, source):
    # the headline step's resampling at its own size: N = M = 2^24, 32-byte
    # particle records, the maximum taken from the trace kernel's summary as
    # in the timed step; "linefitting" resamples the trace kernel's own
    # population (256 points, ESS near 1: most outputs share a few ancestors),
    # "normal" a population with ESS near N/e (unit-variance log-weights: the
    # merge path's many-ancestor case); ancestors and records bit for bit
    import torch
    N = 1 << 24
    model = ppl.poly_model()
    parts = ppl.poly_particles(N)
    if source == "linefitting":
        x, y = synth.poly_dataset(256, 1)
        lw = torch.empty(N, dtype=torch.float32, device="cuda")
        res = ppl.ppl_infer_is_instance(model, _t(x), _t(y), N, 1, 0, lw_out=lw,
                                        particles_out=parts)
        mx = ppl.result_max_lw(res)
    else:
        lw = _t(synth.log_weights(N, 21, "normal", scale=1.0))
        rng = np.random.default_rng(5)
        parts.copy_(torch.from_numpy(rng.standard_normal((N, 8)).astype(np.float32)))
        mx = None
    anc, out = ppl.ppl_resample_gather(N, 1, lw, parts, max_lw_dev=mx, instance=0, t=0)
    lw_h, parts_h = lw.cpu().numpy(), parts.cpu().numpy()
    st, anc_ref = orc.resample_from_lw(lw_h, N, 1, 0, 0)
    assert st == 0
    anc_h = anc.cpu().numpy()
    assert np.array_equal(anc_h, anc_ref)
    assert np.array_equal(out.cpu().numpy().view(np.uint32),
                          orc.gather(parts_h, anc_ref).view(np.uint32))
    if source == "normal":
        assert len(np.unique(anc_h)) > N // 4  # many distinct ancestors
