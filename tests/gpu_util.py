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
    assert np.allclose(res["p_n"], ref["p_n"], rtol=1e-4, atol=1e-12)
    scale = np.max(np.abs(ref["mean_c"])) + 1e-12
    assert np.allclose(res["mean_c"], ref["mean_c"], rtol=1e-4, atol=1e-5 * scale)
    for d in range(ref["n_deg"]):
        if ref["deg_argmax"][d] < 0:
            continue
        dm, dr = res["deg_mean"][d], ref["deg_mean"][d]
        s = np.max(np.abs(dr)) + 1e-12
        assert np.allclose(dm, dr, rtol=1e-4, atol=1e-5 * s), (d, dm, dr)
        second = dr ** 2 + ref["deg_var"][d]
        assert np.all(np.abs(res["deg_var"][d] - ref["deg_var"][d])
                      <= 1e-3 * ref["deg_var"][d] + 1e-6 * second + 1e-9), d
    assert res["map_deg"] == ref["map_deg"] or \
        abs(ref["p_n"][res["map_deg"] - 2] - ref["p_n"][ref["map_deg"] - 2]) < 1e-6
    return ref


