"""Splitting the pair sums over several devices, one process per GPU.

Two partitions of the work, both exact:

* Row blocks of one operator application.  Every rank holds the whole point
  set and the whole density, evaluates the targets of its own contiguous
  block of the spatial (layout) order with ``ssd_apply_rows``, and one
  all-reduce of the zero-filled results assembles the application on every
  rank (adding zeros is exact, so the result is bit-identical to the
  one-device application on the direct kernels, and equal to the rounding
  of the precision where the one-device application runs a symmetric
  plan).  Compute is O(N^2 / P) per rank against O(N) exchanged.
* Surfaces of a batch.  Independent problems: each rank takes a set of
  surfaces, balanced by their pair counts, and nothing is exchanged until the
  results are gathered.

The functions below hold only the partition logic and the exchange; the
arithmetic of every step runs in the library (``apply_rows``) or, in the
CPU tests, in a stand-in with the same signature.
"""
from __future__ import annotations

import numpy as np

ROW_ALIGN = 512   # target tile of the pair kernels: blocks start on tile boundaries


def row_blocks(n: int, world: int, align: int = ROW_ALIGN):
    """[(begin, end)] of `world` contiguous row blocks covering [0, n): the
    boundaries are r n / world rounded to a multiple of `align`, so every
    block is within `align` of n / world (a block may be empty when n is
    small)."""
    if n <= 0 or world <= 0:
        raise ValueError("n and world must be positive")
    cuts = [0] + [min(n, int(round(r * n / (world * align))) * align) for r in range(1, world)] + [n]
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def surface_blocks(sizes, world: int):
    """Surfaces per rank, balanced by pair count n_s^2: largest first to the
    least-loaded rank (ties to the lower rank).  Returns a list of index lists."""
    if world <= 0:
        raise ValueError("world must be positive")
    load = [0] * world
    out = [[] for _ in range(world)]
    for s in sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]) ** 2, k)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(s)
        load[r] += int(sizes[s]) ** 2
    return [sorted(v) for v in out]


def sharded_apply(apply_rows, n: int, rank: int, world: int, all_reduce, align: int = ROW_ALIGN):
    """One operator application split into row blocks.

    apply_rows(b, e) returns a full-size array with the rows [b, e) of the
    spatial order filled and every other entry zero; all_reduce(x) sums x
    over the ranks in place.  Returns the whole application on every rank.
    """
    b, e = row_blocks(n, world, align)[rank]
    out = apply_rows(b, e)
    all_reduce(out)
    return out


def device_apply_sharded(ctx, pts, op, delta, dens, mu=1.0, prec=None, group=None):
    """sharded_apply on the device: ``ssd_apply_rows`` for this rank's rows
    and a torch.distributed all-reduce (NCCL on GPUs) of the zero-filled
    result.  Without a process group it is the whole application."""
    import torch.distributed as dist

    import paper_2110_10749_gb300 as ssd
    prec = ssd.FP64 if prec is None else prec
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0

    def rows(b, e):
        if e <= b:
            import torch
            return torch.zeros_like(dens)
        return ssd.apply_rows(ctx, pts, op, delta, dens, b, e, mu=mu, prec=prec)

    def reduce(x):
        if world > 1:
            dist.all_reduce(x, group=group)
    return sharded_apply(rows, pts.n, rank, world, reduce)
