"""Host logic of a population split over ranks, as gloo ranks on CPU (no GPU).

Every rank holds the same seeded log-weights; the oracle's fixed-point
weights of the whole population stand in for the device shard sums.  The
shards' sums are all-gathered, the library's host planner
(ppl_resample_shard_plan) turns them into each shard's outputs, and those
must partition the oracle's unsplit ancestors exactly: shard g's outputs are
those whose ancestor lies in g's particle range.  The rebalancing exchange
then moves each shard's outputs to their owning ranks by point-to-point
messages, which must reproduce the oracle's ancestors row for row.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q, n, m, kind, seed):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle
    import synth
    from paper_2010_08454_gb300 import binding as ppl
    from paper_2010_08454_gb300 import sharded
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                                world_size=world)
        lw = synth.log_weights(n, seed, kind)
        q_all = oracle.quantize_weights(lw)  # the population's fixed-point weights
        first, end = sharded.shard_range(n, rank, world)
        total = torch.tensor([int(q_all[first:end].sum(dtype=np.uint64))], dtype=torch.int64)
        totals = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(totals, total)
        sums = np.array([int(t.item()) for t in totals], dtype=np.uint64)
        plans = ppl.ppl_resample_shard_plan(sums, n, m, seed, 1, 2)
        st, anc = oracle.resample_systematic(q_all, m, seed, 1, 2)
        assert st == 0
        plan = plans[rank]
        bounds = [p.k_first for p in plans] + [plans[-1].k_end]
        # the shard's outputs are exactly those descending from its particles
        mine = anc[plan.k_first:plan.k_end]
        assert np.all((mine >= first) & (mine < end))
        assert plan.k_first == int(np.searchsorted(anc, first, side="left"))
        assert plan.k_end == int(np.searchsorted(anc, end, side="left"))
        held = torch.from_numpy(mine.astype(np.int64))
        owned = sharded.rebalance(held, plan.k_first, bounds, m)
        o0, o1 = sharded.shard_range(m, rank, world)
        assert np.array_equal(owned.numpy(), anc[o0:o1].astype(np.int64))
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, "ok", bounds))
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, f"{type(e).__name__}: {e}", None))


@pytest.mark.parametrize("world,n,m,kind", [(2, 100003, 77777, "normal"),
                                            (2, 65536, 65536, "onehot"),
                                            (3, 50000, 120001, "sparse"),
                                            (3, 4099, 4099, "wide")])
def test_shard_plan_and_rebalance_reproduce_unsplit_ancestors(world, n, m, kind):
    sys.path.insert(0, ROOT)
    from paper_2010_08454_gb300 import build
    build.build()  # once, before the ranks load the library
    port = _free_port()
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, n, m, kind, 11 + world))
             for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
    for rank, msg, bounds in out:
        assert msg == "ok", (rank, msg)
    # every rank computed the same plan, covering all outputs in order
    assert all(b == out[0][2] for _, _, b in out)
    assert out[0][2][0] == 0 and out[0][2][-1] == m


def test_exchange_plan_covers_every_output_once():
    sys.path.insert(0, ROOT)
    from paper_2010_08454_gb300 import sharded
    bounds, m, world = [0, 0, 9, 9, 20], 20, 4
    moves = sharded.exchange_plan(bounds, m, world)
    seen = np.zeros(m, dtype=int)
    for src, dst, k0, k1 in moves:
        assert bounds[src] <= k0 < k1 <= bounds[src + 1]
        d0, d1 = sharded.shard_range(m, dst, world)
        assert d0 <= k0 and k1 <= d1
        seen[k0:k1] += 1
    assert np.all(seen == 1)
