"""Neutron-id shards of a multi-GPU run and the one exchange step of the path.

Rank r of w traces the ids first_id + [r n, (r + 1) n) of the same random stream (seed,
sim_id).  A neutron's history depends only on (seed, sim_id, id), so the histograms and
tallies of the ranks add up to those of one run over the union of the ranges (up to the order
of the FP64 additions).  The forward path needs no exchange until its result is wanted: one
sum over the ranks of the FP64 histograms and tallies (reduce_sum).

The gradient of the chi-squared loss does exchange data on its way: the loss and its
derivative dchi2/dI are functions of the WHOLE run's histogram, so the ranks sum their
forward histograms before the adjoint, and sum the per-rank gradients after it
(sharded_gradient).  On GPUs the sums run over NCCL, on host tensors over gloo.
"""
from __future__ import annotations


def shard(rank: int, world: int, n_per_rank: int, first_id: int = 0):
    """(first id, count) of `rank` when every rank traces n_per_rank neutrons."""
    if not (0 <= rank < world) or n_per_rank < 0 or first_id < 0:
        raise ValueError("bad shard request")
    return first_id + rank * n_per_rank, n_per_rank


def split(rank: int, world: int, n_total: int, first_id: int = 0):
    """(first id, count) of `rank` when n_total neutrons are divided over the ranks (strong
    scaling): contiguous ranges whose sizes differ by at most one."""
    if not (0 <= rank < world) or n_total < 0 or first_id < 0:
        raise ValueError("bad split request")
    lo = (n_total * rank) // world
    hi = (n_total * (rank + 1)) // world
    return first_id + lo, hi - lo


def reduce_sum(tensors, group=None, dst=None):
    """Sums each tensor over the ranks of `group`, in place: on every rank (all_reduce), or
    only on rank `dst` (reduce; the other ranks' tensors are then unspecified).  A no-op when
    torch.distributed is not initialised (one process)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return tensors
    for t in tensors:
        if t is None:
            continue
        if dst is None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        else:
            dist.reduce(t, dst, op=dist.ReduceOp.SUM, group=group)
    return tensors


def sharded_gradient(forward, adjoint, hist, rank, world, n_total, first_id=0, group=None):
    """The loss of a run split over the ranks and its gradient.

    forward(first, n, hist) adds the forward histogram of ids first..first+n-1 into `hist`
    (zeroed by the caller); adjoint(first, n, hist) returns {"loss", "dsqe", "dsig"}: the loss
    of the histogram `hist` and the gradient of those ids only (mcv_adjoint on a GPU).  Steps:
    this rank's forward, the sum of the histograms (every rank then holds the whole run's),
    this rank's adjoint, and the sum of the gradients.  Returns the adjoint's dict with the
    summed gradient (the same on every rank) and `hist`, the whole run's histogram."""
    first, n = split(rank, world, n_total, first_id)
    forward(first, n, hist)
    reduce_sum([hist], group)
    out = adjoint(first, n, hist)
    reduce_sum([out["dsqe"], out["dsig"]], group)
    out["hist"] = hist
    return out
