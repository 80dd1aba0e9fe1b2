"""Pins for the oracle's fixed-point systematic resampling and gather.

Ancestors are checked against a brute-force search written with the library's
searchsorted over numpy cumulative sums, and against the invariants every
systematic resampler satisfies; the FP32 exponential that decides the integer
weights is checked against FP64 exp.
"""
import numpy as np
import pytest

import synth


def test_exp32_accuracy(orc):
    d = np.concatenate([np.linspace(-44.5, 0, 20001), -np.logspace(-8, 1.6, 2000)])
    d = d.astype(np.float32)
    got = np.array([orc.exp32(v) for v in d], dtype=np.float64)
    ref = np.exp(d.astype(np.float64))
    assert np.max(np.abs(got / ref - 1)) < 3 * 2.0 ** -24
    assert orc.exp32(0.0) == 1.0
    assert all(orc.exp32(v) <= 1.0 for v in d)


def test_fixed_shift(orc):
    assert orc.fixed_shift(1) == 61
    assert orc.fixed_shift(2) == 60
    assert orc.fixed_shift(3) == 59
    assert orc.fixed_shift(1 << 24) == 37
    assert orc.fixed_shift((1 << 24) + 1) == 36


@pytest.mark.parametrize("kind", ["normal", "equal", "onehot", "sparse", "wide"])
def test_quantize_weights(orc, kind):
    N = 3001
    lw = synth.log_weights(N, 3, kind)
    q = orc.quantize_weights(lw)
    S = orc.fixed_shift(N)
    d = (lw - lw.max()).astype(np.float64)
    ideal = np.where(d >= -44.5, np.exp(d) * 2.0 ** S, 0.0)
    ok = ideal >= 2.0 ** 30
    assert np.all(np.abs(q[ok].astype(np.float64) / ideal[ok] - 1) < 3 * 2.0 ** -24)
    assert np.all(q[~ok].astype(np.float64) <= ideal[~ok] * (1 + 1e-6) + 1)
    assert q.max() == np.uint64(1) << np.uint64(S)
    assert int(q.astype(object).sum()) <= 2 ** 61


def _offset(orc, seed, instance, step_t, stride):
    w = int(orc.philox_block(seed, 0, instance, step_t, 3, 0)[0])
    return (w * stride) >> 32


@pytest.mark.parametrize("N,M", [(1, 1), (2, 5), (17, 17), (100, 37), (257, 1000), (1000, 1000)])
def test_systematic_matches_brute_force(orc, N, M):
    for seed in range(3):
        q = synth.fixed_weights(N, seed)
        if q.sum() == 0:
            q[0] = 5
        st, anc = orc.resample_systematic(q, M, seed, 2, 9)
        assert st == 0
        T = int(q.astype(object).sum())
        step = T // M
        u = _offset(orc, seed, 2, 9, step)
        C = np.cumsum(q.astype(object))
        ref = [next(j for j in range(N) if C[j] > u + k * step) for k in range(M)]
        assert np.array_equal(anc, ref)


@pytest.mark.parametrize("kind", ["normal", "equal", "onehot", "sparse", "wide"])
def test_systematic_invariants(orc, kind):
    N = M = 4099
    lw = synth.log_weights(N, 8, kind)
    q = orc.quantize_weights(lw)
    st, anc = orc.resample_systematic(q, M, 1, 0, 3)
    assert st == 0
    assert np.all(np.diff(anc) >= 0)                 # ancestors are monotone
    off = np.bincount(anc, minlength=N)
    assert off.sum() == M
    assert np.all(off[q == 0] == 0)                  # zero weight is never chosen
    step = int(q.astype(object).sum()) // M
    expect = q.astype(np.float64) / step
    assert np.all(np.abs(off - expect) < 1 + 1e-9)   # |o_j - q_j / step| < 1
    st2, anc2 = orc.resample_from_lw(lw, M, 1, 0, 3)
    assert st2 == 0 and np.array_equal(anc, anc2)


def test_equal_weights_keep_every_particle(orc):
    N = 1000
    q = np.full(N, 12345, dtype=np.uint64)
    st, anc = orc.resample_systematic(q, N, 4, 0, 0)
    assert st == 0 and np.array_equal(anc, np.arange(N))


def test_resample_errors(orc):
    st, _ = orc.resample_systematic(np.zeros(10, dtype=np.uint64), 10, 0)
    assert st == 5
    st, _ = orc.resample_systematic(np.full(10, 1, dtype=np.uint64), 11, 0)
    assert st == 1
    lw = np.zeros(4, dtype=np.float32)
    lw[2] = np.nan
    st, _ = orc.resample_from_lw(lw, 4, 0)
    assert st == 4


def test_gather(orc):
    rec = np.arange(40, dtype=np.float32).reshape(5, 8)
    anc = np.array([0, 0, 3, 4, 4, 4], dtype=np.int32)
    out = orc.gather(rec, anc)
    assert np.array_equal(out, rec[anc])
