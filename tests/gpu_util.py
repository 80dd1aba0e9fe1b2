"""Helpers shared by the GPU parity tests: marshalling, and the comparison of a
likelihood-weighting result with the oracle (no arithmetic of the method)."""
import numpy as np
import pytest


def load_ppl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_08454_gb300 as ppl
    ppl.lib()
    return ppl


def gpu_is(ppl, x, y, N, seed, fn=None, **model_kw):
    import torch
    model = ppl.poly_model(**model_kw)
    fn = fn or ppl.ppl_infer_is
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).cuda()
    lw = torch.empty(N, dtype=torch.float32, device="cuda")
    parts = ppl.poly_particles(N)
    ws = ppl.workspace(model, N, len(x))
    res = ppl.read_result(fn(model, xd, yd, N, seed, lw_out=lw, particles_out=parts, ws=ws))
    c, n, origin = ppl.decode_particles(parts)
    return res, lw.cpu().numpy(), n.cpu().numpy(), c.cpu().numpy(), origin.cpu().numpy()


def check_is(orc, res, lw, n, c, origin, x, y, N, seed, model_kw, full=True):
    """A GPU likelihood-weighting result against the FP64 oracle at equal seeds:
    discrete draws bit-exact; coefficients and log-weights within the FP32
    error of the traces; |delta log Z| <= 1e-3 (plus four FP32 ulps of the
    largest log-weight, which only matters when |max lw| > 1000); degree masses
    and weighted coefficient means within 1e-4 relative."""
    om = orc.poly_model(**model_kw)
    ref, (lw_r, n_r, c_r) = orc.infer_is_poly(om, x, y, N, seed)
    assert res["status"] == 0
    assert np.array_equal(n, n_r)                                  # discrete draws: exact
    assert np.array_equal(origin, np.arange(N))
    assert np.allclose(c, c_r, rtol=1e-5, atol=1e-4)              # FP32 Box-Muller
    err = np.abs(lw.astype(np.float64) - lw_r)
    assert np.all(err <= 4e-6 * np.abs(lw_r) + 1e-3), float(np.max(err - 4e-6 * np.abs(lw_r)))
    # 1e-3, widened by four FP32 ulps of the largest log-weight for data sets
    # whose log-weights are so large that FP32 cannot resolve 1e-3
    assert abs(res["log_z"] - ref["log_z"]) <= 1e-3 + 2.0 ** -21 * abs(ref["max_lw"])
    assert res["ess"] == pytest.approx(ref["ess"], rel=1e-3)
    assert res["max_lw"] == pytest.approx(ref["max_lw"], rel=4e-6, abs=1e-3)
    if res["argmax"] != ref["argmax"]:  # a near-tie may order differently in FP32
        assert abs(lw_r[res["argmax"]] - ref["max_lw"]) <= 4e-6 * abs(ref["max_lw"]) + 1e-3
    check_summary(res, ref)
    return ref


def lw_resolution(max_lw):
    """FP32 resolution of the log-weights that carry a population's weight: at
    most 4e-6 relative per trace (the per-trace bound the trace tests assert;
    measured at most 8.1e-7), taken at |max lw| + 50 because traces more than
    50 nats below the maximum carry less than e^-50 of the weight."""
    return 4e-6 * (np.abs(max_lw) + 50.0)


def check_summary(res, ref, where=None):
    """The posterior summary of one population against the oracle's.

    Every moment must agree within 1e-4 relative, widened only by what the
    FP32 log-weights themselves leave undetermined.  A per-trace log-weight
    error delta_i (|delta_i| <= eps, eps = lw_resolution of the traces that
    carry weight) moves normalised weights by the factor exp(delta_i - mean
    delta), so to first order a weighted mean moves by Cov_W(delta, c), at
    most eps * sd_W(c), and a degree mass p_n by a relative
    mean_n(delta) - mean(delta), at most eps_n + eps_max.  Hence:
      p_n:        1e-4 p_n + (eps_n + eps_max) p_n
      deg_mean:   1e-4 |mean| + 1e-5 max|mean of the degree| + 2 eps_n sd
      deg_var:    (1e-3 + 4 eps_n) var + 1e-6 second moment
      mean_c:     1e-4 |mean_c| + 1e-5 max|mean_c| + sum_n (p_n tol |mean_n| + 2 p_n eps_n sd_n)
    The eps terms vanish for well-fitting data (|lw| of tens: eps < 4e-4)
    and matter only for degrees whose best trace lies hundreds of nats below
    zero, whose mass is then negligible.  The MAP degree must be equal unless
    the two masses tie within 1e-6."""
    nd = ref["n_deg"]
    has = np.array([ref["deg_argmax"][d] >= 0 for d in range(4)])
    eps_d = np.where(has, lw_resolution(np.where(has, ref["deg_max_lw"], 0.0)), 0.0)
    eps_max = lw_resolution(ref["max_lw"])
    p, pr = np.asarray(res["p_n"]), np.asarray(ref["p_n"])
    tol_p = 1e-4 * pr + (eps_d + eps_max) * pr + 1e-300
    assert np.all(np.abs(p - pr) <= tol_p), (where, p, pr, tol_p)
    sd = np.sqrt(np.maximum(ref["deg_var"], 0.0))
    for d in range(nd):
        if not has[d]:
            continue
        dm, dr = res["deg_mean"][d], ref["deg_mean"][d]
        tol = 1e-4 * np.abs(dr) + 1e-5 * (np.max(np.abs(dr)) + 1e-12) + 2 * eps_d[d] * sd[d]
        assert np.all(np.abs(dm - dr) <= tol), (where, d, dm, dr, tol)
        second = dr ** 2 + ref["deg_var"][d]
        tol_v = (1e-3 + 4 * eps_d[d]) * ref["deg_var"][d] + 1e-6 * second + 1e-9
        assert np.all(np.abs(res["deg_var"][d] - ref["deg_var"][d]) <= tol_v), \
            (where, d, res["deg_var"][d], ref["deg_var"][d])
    mr = ref["mean_c"]
    tol_c = 1e-4 * np.abs(mr) + 1e-5 * (np.max(np.abs(mr)) + 1e-12)
    for d in range(nd):
        if has[d]:
            tol_c = tol_c + tol_p[d] * np.abs(ref["deg_mean"][d]) + 2 * pr[d] * eps_d[d] * sd[d]
    assert np.all(np.abs(res["mean_c"] - mr) <= tol_c), (where, res["mean_c"], mr, tol_c)
    assert res["map_deg"] == ref["map_deg"] or \
        abs(ref["p_n"][res["map_deg"] - 2] - ref["p_n"][ref["map_deg"] - 2]) < 1e-6, where
