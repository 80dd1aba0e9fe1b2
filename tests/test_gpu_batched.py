"""Parity of the batched persistent launch with the oracle, instance by
instance, plus graph replay and the autotuner's cache."""
import json
import os

import numpy as np
import pytest

import synth
from gpu_util import check_summary, load_ppl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppl():
    return load_ppl()


def _device_batch(ppl, inst):
    import torch
    return (torch.from_numpy(inst["x"]).cuda(), torch.from_numpy(inst["y"]).cuda(),
            torch.from_numpy(inst["data_off"]).cuda(), torch.from_numpy(inst["part_off"]).cuda())


def _check_instances(orc, inst, results, seed, which):
    om = orc.poly_model()
    for b in which:
        d0, d1 = inst["data_off"][b], inst["data_off"][b + 1]
        N = int(inst["N"][b])
        ref, _ = orc.infer_is_poly(om, inst["x"][d0:d1], inst["y"][d0:d1], N, seed, instance=b)
        r = results[b]
        assert r["status"] == 0 and r["n_particles"] == N
        tol = 1e-3 + 2.0 ** -21 * abs(ref["max_lw"])  # 4 FP32 ulps of the largest lw
        assert abs(r["log_z"] - ref["log_z"]) <= tol, (b, r["log_z"], ref["log_z"])
        assert r["ess"] == pytest.approx(ref["ess"], rel=1e-3)
        check_summary(r, ref, b)
        if r["argmax"] != ref["argmax"]:
            assert abs(r["max_lw"] - ref["max_lw"]) <= tol


@pytest.mark.parametrize("ppt,bps", [(1, 1), (4, 2), (8, 4)])
def test_batched_matches_oracle_per_instance(ppl, orc, ppt, bps):
    inst = synth.batched_instances(40, 77, L_range=(1, 9000), N_range=(1, 5000))
    x, y, doff, poff = _device_batch(ppl, inst)
    model = ppl.poly_model()
    ws = ppl.batched_workspace(inst["data_off"], inst["part_off"])
    plan = ppl.ppl_batched_prepare(model, inst["data_off"], inst["part_off"], ppt, bps, ws)
    out = ppl.batch_results_tensor(40)
    ppl.ppl_infer_is_batched(model, x, y, doff, poff, 13, plan, out, ws)
    assert ppl.ppl_batched_status(ws) == 0
    res = ppl.read_batch_results(out, 40)
    _check_instances(orc, inst, res, 13, range(40))


def test_graph_replay_and_autotune_cache(ppl, orc, tmp_path):
    import torch
    inst = synth.batched_instances(300, 3, N_range=(2 ** 8, 2 ** 12))
    x, y, doff, poff = _device_batch(ppl, inst)
    model = ppl.poly_model()
    ws = ppl.batched_workspace(inst["data_off"], inst["part_off"])
    out = ppl.batch_results_tensor(300)
    cache = str(tmp_path / "batched_tune.json")
    plan = ppl.ppl_batched_autotune(model, x, y, doff, poff, inst["data_off"], inst["part_off"],
                                    5, out, ws, cache)
    assert plan.ppt in (1, 2, 4, 8) and 1 <= plan.blocks_per_sm <= 4
    entry = json.loads(open(cache).read())
    assert entry["ppt"] == plan.ppt and entry["blocks_per_sm"] == plan.blocks_per_sm
    again = ppl.ppl_batched_autotune(model, x, y, doff, poff, inst["data_off"],
                                     inst["part_off"], 5, out, ws, cache)
    assert (again.ppt, again.blocks_per_sm) == (plan.ppt, plan.blocks_per_sm)
    # capture the launch in a CUDA graph and replay it
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ppl.ppl_infer_is_batched(model, x, y, doff, poff, 5, plan, out, ws)
    out.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    res = ppl.read_batch_results(out, 300)
    _check_instances(orc, inst, res, 5, list(range(0, 300, 23)) + [299])


def test_batched_4096_instances_sampled_against_oracle(ppl, orc, tmp_path):
    # the benchmarked shape itself: 4096 instances, data lengths log-uniform in
    # [16, 4096], particle counts log-uniform in [2^10, 2^16], one autotuned
    # launch; 48 instances checked against the oracle: the eight largest N x L,
    # the largest N (tens of tiles, where the running maxima of earlier tiles
    # decide which traces later tiles skip), the largest and
    # smallest L, the smallest N, and a seeded draw of the rest
    inst = synth.batched_instances(4096, 3)
    x, y, doff, poff = _device_batch(ppl, inst)
    model = ppl.poly_model()
    ws = ppl.batched_workspace(inst["data_off"], inst["part_off"])
    out = ppl.batch_results_tensor(4096)
    plan = ppl.ppl_batched_autotune(model, x, y, doff, poff, inst["data_off"], inst["part_off"],
                                    3, out, ws, str(tmp_path / "tune.json"))
    out.zero_()
    ppl.ppl_infer_is_batched(model, x, y, doff, poff, 3, plan, out, ws)
    assert ppl.ppl_batched_status(ws) == 0
    res = ppl.read_batch_results(out, 4096)
    N, L = inst["N"], inst["L"]
    pick = {int(b) for b in np.argsort(N * L)[-8:]}
    pick |= {int(np.argmax(N)), int(np.argmax(L)), int(np.argmin(L)), int(np.argmin(N))}
    rest = np.setdiff1d(np.arange(4096), sorted(pick))
    pick |= {int(b) for b in np.random.default_rng(48).choice(rest, 48 - len(pick), replace=False)}
    pick = sorted(pick)
    assert len(pick) == 48 and max(N[pick]) > 65000
    _check_instances(orc, inst, res, 3, pick)
