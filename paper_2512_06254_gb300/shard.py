"""Sharding one observation's snapshot stream across ranks (one process per
GPU).

S1-S6 are independent per snapshot; the tLISI output at t needs the images
t-2, t-1 and t (S7, Section 2 and Section 4.5: three consecutive images).  An
observation of S snapshots has tLISI outputs t = 2..S-1; they are split into
contiguous blocks, and rank r images snapshots [lo_r - 2, hi_r) so that its
first two images are a halo it recomputes itself: no image crosses ranks.
The candidate search (S8) needs the whole cube, so the tLISI slices are
gathered to every rank (one all-gather of (S-2) x (N/T)^2 float32, 16 KB per
slice at 64 x 64 tiles): the single collective of the path.

This module holds the host logic only; the per-snapshot work is whatever
`image_and_tlisi` does (the library's plan in bench.py, anything in tests).
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import torch


def tlisi_range(S: int, world: int, rank: int) -> Tuple[int, int]:
    """tLISI outputs [lo, hi) owned by `rank`: the S - 2 outputs t = 2..S-1
    in contiguous blocks whose sizes differ by at most one (empty when
    there are fewer outputs than ranks)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    n = max(S - 2, 0)
    base, extra = divmod(n, world)
    lo = 2 + rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def image_range(S: int, world: int, rank: int) -> Tuple[int, int]:
    """Snapshots [first, hi) that `rank` images: its outputs' three-image
    windows, i.e. [lo - 2, hi); empty when it owns no output."""
    lo, hi = tlisi_range(S, world, rank)
    if hi <= lo:
        return lo, lo
    return lo - 2, hi


def run_shard(S: int, world: int, rank: int,
              image_and_tlisi: Callable[[int, Optional[torch.Tensor]], bool],
              out: torch.Tensor) -> Tuple[int, int]:
    """Image this rank's snapshots in order.  `image_and_tlisi(s, dst)`
    images snapshot s, pushes it into the plan's three-image ring and writes
    the tLISI of the ring into dst (a [nty, ntx] view of `out`) when it
    returns True (the ring is full).  `out` has at least hi - lo slices;
    slice i receives output t = lo + i.  Returns (lo, hi)."""
    first, hi = image_range(S, world, rank)
    lo, _ = tlisi_range(S, world, rank)
    for s in range(first, hi):
        dst = out[s - lo] if s >= lo else None
        valid = image_and_tlisi(s, dst)
        if valid != (s >= lo):
            raise RuntimeError(f"snapshot {s}: tLISI validity {valid}, expected {s >= lo}")
    return lo, hi


def run_shard_batched(S: int, world: int, rank: int,
                      image_batch: Callable[[int, int, int], int], batch: int) -> Tuple[int, int]:
    """Image this rank's snapshots [lo - 2, hi) in order, in batches of at
    most `batch` (the library's batched engine).  `image_batch(s0, s1, row)`
    images snapshots [s0, s1) as the next batch of the plan's stream and
    returns its first_valid (the entries before it have no three-image
    window yet); the tLISI of snapshot s >= lo belongs in local row s - lo,
    and `row` = s0 - lo is the local row of the batch's first snapshot
    (negative for the 2-snapshot halo, whose entries get no tLISI).
    Returns (lo, hi)."""
    if batch < 1:
        raise ValueError("batch must be >= 1")
    first, hi = image_range(S, world, rank)
    lo, _ = tlisi_range(S, world, rank)
    for s0 in range(first, hi, batch):
        s1 = min(hi, s0 + batch)
        fv = image_batch(s0, s1, s0 - lo)
        expected = max(0, min(lo - s0, s1 - s0))
        if fv != expected:
            raise RuntimeError(f"batch [{s0}, {s1}): first_valid {fv}, expected {expected}")
    return lo, hi


def gather_cube(local: torch.Tensor, S: int, world: int, rank: int, group=None) -> torch.Tensor:
    """All-gather the ranks' tLISI blocks into the full cube [S - 2, nty, ntx]
    (same device as `local`).  `local` holds this rank's hi - lo slices in its
    first rows and at least ceil((S - 2) / world) rows in total."""
    import torch.distributed as dist
    width = -(-max(S - 2, 0) // world)
    if local.shape[0] < width:
        raise ValueError("local cube has fewer rows than the largest block")
    send = local[:width].contiguous()
    if world == 1:
        parts = [send]
    else:
        parts = [torch.empty_like(send) for _ in range(world)]
        dist.all_gather(parts, send, group=group)
    blocks = []
    for r in range(world):
        lo, hi = tlisi_range(S, world, r)
        blocks.append(parts[r][:hi - lo])
    return torch.cat(blocks, dim=0)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest `value` over all ranks (the bench's step time)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
