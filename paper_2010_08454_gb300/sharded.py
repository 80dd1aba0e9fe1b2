"""One population of particles split over several ranks (one GPU each).

Particle methods scale out (the paper names them as future work, §6): the
traces are independent, and normalisation (§3.6.2) and resampling need only
a few numbers from every rank.  This module is the host-side plumbing that
connects the library's shard entry points with torch.distributed; every
step of the method itself runs in libppl.so.

* Likelihood weighting: rank r draws the particles of its contiguous range of
  the global index (the same traces as the unsplit call), reduces them to a
  384-byte partial, and an all-gather of the partials feeds one merge.
* Systematic resampling: an all-reduce gives the population's maximum
  log-weight, an all-gather the shards' sums of fixed-point weights; every
  rank then computes the same plan, and each resamples its own outputs
  (their ancestors are all its own particles).  Rebalancing moves those
  outputs to the ranks that own them after resampling (rank r owns outputs
  [r m / W, (r + 1) m / W)) by point-to-point exchange of contiguous ranges.
"""
import numpy as np
import torch
import torch.distributed as dist

from . import binding as ppl


def shard_range(n_total, rank, world):
    """Rank `rank`'s contiguous share [first, end) of n_total particles."""
    return n_total * rank // world, n_total * (rank + 1) // world


def infer_is_sharded(model, x, y, n_total, seed, instance=0, group=None, lw_out=None,
                     particles_out=None, ws=None, out=None):
    """Likelihood weighting of n_total particles over the ranks of `group`:
    every rank returns the population's summary (device ppl_is_result)."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    first, end = shard_range(n_total, rank, world)
    part = ppl.ppl_infer_is_partial(model, x, y, first, end - first, seed, instance,
                                    lw_out=lw_out, particles_out=particles_out, ws=ws)
    gathered = ppl.partial_tensor(world, part.device)
    dist.all_gather_into_tensor(gathered.view(-1), part.view(-1), group=group)
    return ppl.ppl_is_merge(gathered, out=out)


def exchange_plan(k_bounds, m, world):
    """Which contiguous output ranges move between ranks when the outputs
    [k_bounds[g], k_bounds[g + 1]) held by rank g go to their owners (rank r
    owns [r m / W, (r + 1) m / W)): a list of (src, dst, k0, k1)."""
    moves = []
    for src in range(world):
        a0, a1 = int(k_bounds[src]), int(k_bounds[src + 1])
        for dst in range(world):
            b0, b1 = shard_range(m, dst, world)
            k0, k1 = max(a0, b0), min(a1, b1)
            if k0 < k1:
                moves.append((src, dst, k0, k1))
    return moves


def rebalance(held, k_first, k_bounds, m, group=None):
    """Move this rank's outputs `held` (rows k_first .. of the population's
    outputs) to their owners; returns this rank's owned rows."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    o0, o1 = shard_range(m, rank, world)
    owned = torch.empty((o1 - o0,) + tuple(held.shape[1:]), dtype=held.dtype,
                        device=held.device)
    reqs = []
    for src, dst, k0, k1 in exchange_plan(k_bounds, m, world):
        if src == rank and dst == rank:
            owned[k0 - o0:k1 - o0].copy_(held[k0 - k_first:k1 - k_first])
        elif src == rank:
            reqs.append(dist.isend(held[k0 - k_first:k1 - k_first].contiguous(), dst, group=group))
        elif dst == rank:
            buf = owned[k0 - o0:k1 - o0]
            reqs.append((dist.irecv(buf, src, group=group), buf))
    for r in reqs:
        (r[0] if isinstance(r, tuple) else r).wait()
    return owned


def resample_sharded(lw, n_total, m, seed, instance=0, t=0, state=None, group=None, ws=None,
                     rebalance_outputs=True):
    """Systematic resampling of a population whose log-weights are split over
    the ranks (this rank holds particles shard_range(n_total, rank, W)):
    returns (ancestors, states) of this rank's outputs -- the owned rows
    [r m / W, (r + 1) m / W) when rebalance_outputs, else the rows the shard
    produced [plan.k_first, plan.k_end) -- and the plans of all shards."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    first, end = shard_range(n_total, rank, world)
    stats = ppl.ppl_logsumexp(lw)
    mx = stats[2:3].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX, group=group)
    total = ppl.ppl_resample_shard_total(lw, mx, n_total)
    totals = torch.empty(world, dtype=torch.int64, device=lw.device)
    dist.all_gather_into_tensor(totals, total, group=group)
    plans = ppl.ppl_resample_shard_plan(totals.cpu().numpy().view(np.uint64), n_total, m, seed,
                                        instance, t)
    plan = plans[rank]
    anc, out = ppl.ppl_resample_shard(lw, first, mx, plan, state_in=state, ws=ws)
    if not rebalance_outputs:
        return anc, out, plans
    k_bounds = [p.k_first for p in plans] + [plans[-1].k_end]
    anc = rebalance(anc, plan.k_first, k_bounds, m, group)
    if out is not None:
        out = rebalance(out, plan.k_first, k_bounds, m, group)
    return anc, out, plans
