"""Sharding of one projection set over ranks (one process per GPU).

The method's work splits without exchange: histories are independent and keyed
by their index (the Philox counter holds it), and projections are independent
(the paper assigns projections to GPUs, Sec. II-B).  A rank takes a contiguous
range of histories (`history_range`, for `Context.project_histories`) or of
angles (`angle_range`); the only exchange is the FP64 sum of the partial scatter
tallies (`reduce_images`), which equals the one-GPU image up to the order of the
FP64 additions.  Timing over ranks takes the maximum (`max_time`).

These helpers hold host logic only (index ranges and torch.distributed calls);
they run with any backend, so the multi-rank path is tested with gloo on CPU.
"""

from __future__ import annotations


def _span(n, rank, world):
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    q, r = divmod(n, world)
    begin = rank * q + min(rank, r)
    return begin, q + (1 if rank < r else 0)


def history_range(n_photons, rank, world):
    """(h_begin, h_count) of this rank's contiguous share of the histories 0 .. n_photons-1
    (sizes differ by at most one)."""
    return _span(int(n_photons), rank, world)


def angle_range(n_angles, rank, world):
    """(first angle index, count) of this rank's contiguous share of the projections."""
    return _span(int(n_angles), rank, world)


def reduce_images(images, group=None):
    """Sum the ranks' partial tallies in FP64, in place on every rank; returns the FP64 tensor."""
    import torch
    import torch.distributed as dist

    t = images if images.dtype == torch.float64 else images.double()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def max_time(seconds, device=None, group=None):
    """The maximum of a per-rank duration over all ranks (the job's time)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
