"""The sufficient-statistics evaluation of the line-fitting factor
(ppl_infer_is_suffstat) against the FP64 oracle's point-by-point sum, with the
tolerances of the direct path, and against the direct CUDA path at equal seeds
(identical draws).  Singular Gram matrices (fewer distinct points than
coefficients) fall back to the point-by-point sum."""
import numpy as np
import pytest

import synth
from gpu_util import check_is, gpu_is, load_ppl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppl():
    return load_ppl()


def _both(ppl, x, y, N, seed, **kw):
    a = gpu_is(ppl, x, y, N, seed, fn=ppl.ppl_infer_is_suffstat, **kw)
    b = gpu_is(ppl, x, y, N, seed, **kw)
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])  # the same traces
    return a, b


@pytest.mark.parametrize("N,L", [(100000, 32), (1 << 20, 256), (4097, 100), (3000, 4097)])
def test_suffstat_matches_oracle(ppl, orc, N, L):
    x, y = synth.poly_dataset(L, 50 + L)
    (res, lw, n, c, origin), (_, lw_d, _, _, _) = _both(ppl, x, y, N, 4)
    check_is(orc, res, lw, n, c, origin, x, y, N, 4, {})
    # against the direct path's FP32 sums: the same bound
    assert np.all(np.abs(lw - lw_d) <= 8e-6 * np.abs(lw_d) + 2e-3)


@pytest.mark.parametrize("L", [0, 1, 2, 5, 6, 7])
def test_suffstat_few_points_and_singular_gram(ppl, orc, L):
    x, y = synth.poly_dataset(L, 70 + L)
    (res, lw, n, c, origin), _ = _both(ppl, x, y, 5000, 6)
    check_is(orc, res, lw, n, c, origin, x, y, 5000, 6, {})


def test_suffstat_repeated_points(ppl, orc):
    x, y = synth.poly_dataset(64, 9)
    x[:] = np.repeat(x[:4], 16)  # four distinct abscissae: G singular past degree 3
    (res, lw, n, c, origin), _ = _both(ppl, x, y, 20000, 8)
    check_is(orc, res, lw, n, c, origin, x, y, 20000, 8, {})


def test_suffstat_other_readings(ppl, orc):
    x, y = synth.poly_dataset(48, 5)
    for kw in [dict(coef_offset=0), dict(min_deg=0, max_deg=3, obs_sigma=2.0, prior_sigma=3.0),
               dict(min_deg=1, max_deg=1)]:
        (res, lw, n, c, origin), _ = _both(ppl, x, y, 20000, 11, **kw)
        check_is(orc, res, lw, n, c, origin, x, y, 20000, 11, kw)
