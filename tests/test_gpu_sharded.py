"""A population split into shards, run shard by shard on one GPU through the
C ABI, against the unsplit calls: the same traces (records and log-weights
bit for bit), the same summary up to merge roundings, and the same ancestors
and gathered records bit for bit.  The torch.distributed plumbing of the
sharded module runs once as a one-rank NCCL group."""
import os
import socket

import numpy as np
import pytest

import synth
from gpu_util import check_summary, load_ppl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppl():
    return load_ppl()


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bounds(n, parts):
    return [n * g // parts for g in range(parts + 1)]


@pytest.mark.parametrize("L,N,parts", [(256, 300007, 3), (32, 100000, 2), (1, 4099, 4)])
def test_sharded_is_matches_unsplit(ppl, orc, L, N, parts):
    import torch
    x, y = synth.poly_dataset(L, 5)
    xd, yd = _t(x), _t(y)
    model = ppl.poly_model()
    lw = torch.empty(N, dtype=torch.float32, device="cuda")
    rec = ppl.poly_particles(N)
    ref = ppl.read_result(ppl.ppl_infer_is_instance(model, xd, yd, N, 9, 3, lw_out=lw,
                                                    particles_out=rec))
    b = _bounds(N, parts)
    partials = ppl.partial_tensor(parts)
    lw_s = torch.empty_like(lw)
    rec_s = torch.empty_like(rec)
    for g in range(parts):
        n = b[g + 1] - b[g]
        ppl.ppl_infer_is_partial(model, xd, yd, b[g], n, 9, 3, partial=partials[g:g + 1],
                                 lw_out=lw_s[b[g]:b[g + 1]], particles_out=rec_s[b[g]:b[g + 1]])
    res = ppl.read_result(ppl.ppl_is_merge(partials))
    # the same traces, bit for bit
    assert torch.equal(lw_s, lw) and torch.equal(rec_s, rec)
    # the same summary: maxima exact, sums up to the order of roundings
    assert res["status"] == 0 and res["n_particles"] == N
    assert res["max_lw"] == ref["max_lw"] and res["argmax"] == ref["argmax"]
    assert np.array_equal(res["deg_max_lw"], ref["deg_max_lw"])
    assert np.array_equal(res["deg_argmax"], ref["deg_argmax"])
    assert res["log_z"] == pytest.approx(ref["log_z"], abs=1e-6)
    assert res["ess"] == pytest.approx(ref["ess"], rel=1e-5)
    check_summary(res, ref, "split vs unsplit")
    # and against the oracle
    oref, _ = orc.infer_is_poly(orc.poly_model(), x, y, N, 9, instance=3)
    assert abs(res["log_z"] - oref["log_z"]) <= 1e-3 + 2.0 ** -21 * abs(oref["max_lw"])
    check_summary(res, oref, "split vs oracle")


@pytest.mark.parametrize("kind", ["normal", "onehot", "sparse"])
@pytest.mark.parametrize("N,M,parts", [(1 << 20, 1 << 20, 3), (300007, 123457, 2),
                                       (4099, 10000, 5)])
def test_sharded_resampling_matches_unsplit(ppl, orc, kind, N, M, parts):
    import torch
    lw_h = synth.log_weights(N, 40 + parts, kind, scale=2.0)
    lw = _t(lw_h)
    rec = _t(np.random.default_rng(N).integers(-99999, 99999, (N, 8)).astype(np.int32))
    anc_ref, rec_ref = ppl.ppl_resample_gather(M, 17, lw, rec, instance=2, t=5)
    b = _bounds(N, parts)
    # 1. the population's maximum from the shards' maxima
    mx = torch.stack([ppl.ppl_logsumexp(lw[b[g]:b[g + 1]])[2] for g in range(parts)]).max()
    mx = mx.reshape(1).clone()
    # 2. the shards' sums, 3. the plans, 4. each shard's outputs
    totals = [int(ppl.ppl_resample_shard_total(lw[b[g]:b[g + 1]], mx, N).item())
              for g in range(parts)]
    plans = ppl.ppl_resample_shard_plan(np.array(totals, dtype=np.uint64), N, M, 17, 2, 5)
    ancs, recs = [], []
    for g in range(parts):
        a, r = ppl.ppl_resample_shard(lw[b[g]:b[g + 1]], b[g], mx, plans[g],
                                      state_in=rec[b[g]:b[g + 1]])
        ancs.append(a)
        recs.append(r)
    assert plans[0].k_first == 0 and plans[-1].k_end == M
    assert torch.equal(torch.cat(ancs), anc_ref)
    assert torch.equal(torch.cat(recs), rec_ref)
    st, ref = orc.resample_from_lw(lw_h, M, 17, 2, 5)
    assert st == 0 and np.array_equal(torch.cat(ancs).cpu().numpy(), ref)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_module_on_a_one_rank_nccl_group(ppl):
    import torch
    import torch.distributed as dist

    from paper_2010_08454_gb300 import sharded
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0,
                            world_size=1)
    try:
        x, y = synth.poly_dataset(256, 1)
        xd, yd = _t(x), _t(y)
        model = ppl.poly_model()
        N = 1 << 18
        lw = torch.empty(N, dtype=torch.float32, device="cuda")
        rec = ppl.poly_particles(N)
        ref = ppl.read_result(ppl.ppl_infer_is_instance(model, xd, yd, N, 4, 0, lw_out=lw,
                                                        particles_out=rec))
        res = ppl.read_result(sharded.infer_is_sharded(model, xd, yd, N, 4))
        assert res["max_lw"] == ref["max_lw"] and res["argmax"] == ref["argmax"]
        assert res["log_z"] == pytest.approx(ref["log_z"], abs=1e-6)
        anc_ref, rec_ref = ppl.ppl_resample_gather(N, 4, lw, rec)
        anc, out, plans = sharded.resample_sharded(lw, N, N, 4, state=rec)
        assert torch.equal(anc, anc_ref) and torch.equal(out, rec_ref)
        torch.cuda.synchronize()
    finally:
        dist.destroy_process_group()
