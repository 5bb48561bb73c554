"""Partitioning of the hot path across processes (one GPU each) and the one
exchange it has: the per-region-pair extremes (Section 3: a brick pair's
indicator is its maximum over point pairs).

Units are independent, so ranks shard them with no data-path collective:

* region pairs (a context view's batched sampling, or any list of region
  pairs): contiguous ranges, `shard_range`;
* the all-pairs refinement of one region pair A x B (Section 4.2): rows of A,
  as sub-boxes whose points are a contiguous range of A's enumeration
  (x fastest, then y, then z), `split_box`. Each rank evaluates its sub-box
  against B; `shift_pair_index` maps its local pair indices to A x B's, and
  `allreduce_extremes` merges the ranks' (max, argmax, min, argmin, count)
  with the same tie rule as one GPU (ties to the smallest linear pair index).
  A self region pair (A == B, only a < b) is sharded at the region-pair level,
  not by rows.

Host logic only; the collective is torch.distributed's all_gather_object
(gloo or NCCL).
"""
from __future__ import annotations

import math


def shard_range(n_units: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) share of n_units for rank (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("need 0 <= rank < world and n_units >= 0")
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def split_box(box, parts: int) -> list[tuple[tuple[int, ...], int]]:
    """Split a half-open box (x0, y0, z0, x1, y1, z1) into at most `parts`
    sub-boxes whose points are contiguous ranges of the box's enumeration.

    Returns [(sub_box, first_index)]: first_index = the sub-box's first point
    in the box's enumeration. Splits along z; along y when the box is one
    layer thick; along x when it is one row. Empty shares are omitted.
    """
    x0, y0, z0, x1, y1, z1 = box
    nx, ny, nz = x1 - x0, y1 - y0, z1 - z0
    if min(nx, ny, nz) <= 0 or parts < 1:
        raise ValueError("empty box or parts < 1")
    if nz > 1:
        axis, n, stride = 2, nz, nx * ny
    elif ny > 1:
        axis, n, stride = 1, ny, nx
    else:
        axis, n, stride = 0, nx, 1
    out = []
    for r in range(parts):
        lo, hi = shard_range(n, r, parts)
        if lo == hi:
            continue
        b = list(box)
        b[axis], b[axis + 3] = box[axis] + lo, box[axis] + hi
        out.append((tuple(b), lo * stride))
    return out


def shift_pair_index(idx: int, first_row: int, nb: int) -> int:
    """Local pair index a_local * nb + b of a sub-box -> the full region pair's."""
    if idx < 0 or idx == 2 ** 64 - 1:
        return idx
    return idx + first_row * nb


_EMPTY = dict(max=-math.inf, min=math.inf, argmax=2 ** 64 - 1, argmin=2 ** 64 - 1, count=0)


def merge_extremes(parts) -> dict:
    """Merge (max, argmax, min, argmin, count) records: larger max wins, ties
    to the smaller argmax; smaller min wins, ties to the smaller argmin."""
    out = dict(_EMPTY)
    for p in parts:
        if p["count"] == 0:
            continue
        if p["max"] > out["max"] or (p["max"] == out["max"] and p["argmax"] < out["argmax"]):
            out["max"], out["argmax"] = p["max"], p["argmax"]
        if p["min"] < out["min"] or (p["min"] == out["min"] and p["argmin"] < out["argmin"]):
            out["min"], out["argmin"] = p["min"], p["argmin"]
        out["count"] += p["count"]
    return out


def allreduce_extremes(local: list[dict], group=None) -> list[dict]:
    """Per-region-pair merge of every rank's records (same region-pair order on
    every rank); returns the merged list on every rank."""
    import torch.distributed as dist
    gathered = [None] * dist.get_world_size(group)
    dist.all_gather_object(gathered, [dict(r) for r in local], group=group)
    if any(len(g) != len(local) for g in gathered):
        raise ValueError("ranks hold different numbers of region pairs")
    return [merge_extremes(g[i] for g in gathered) for i in range(len(local))]


def allgather_shards(local: list, group=None) -> list:
    """Concatenate every rank's shard (rank order) on every rank."""
    import torch.distributed as dist
    gathered = [None] * dist.get_world_size(group)
    dist.all_gather_object(gathered, list(local), group=group)
    return [x for g in gathered for x in g]
