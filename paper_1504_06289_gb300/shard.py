"""Sharding of the Coulomb-matrix and convolution work across ranks.

The path needs no data exchange while it runs: Coulomb-matrix items are
independent (each rank contracts its own items against the same V_H
factors) and factor columns convolve independently.  The only collective is
at the end, to assemble the per-rank results.  One process per GPU; the
helpers below take a torch.distributed process group (NCCL on GPUs, gloo on
CPU) and touch only host-side bookkeeping and the final gather.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def balanced_item_ranges(off: np.ndarray, world: int) -> list:
    """Split items [0, n_items) into `world` contiguous ranges of roughly equal
    factor count (the contraction's cost is proportional to the factor rows, so
    items of uneven CP rank are balanced by rows, not by item count).
    `off` is the item offset array (n_items + 1 entries, nondecreasing)."""
    off = np.asarray(off, dtype=np.int64)
    n_items = len(off) - 1
    total = int(off[-1])
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        bounds.append(int(np.searchsorted(off, target, side="left")))
    bounds.append(n_items)
    bounds = np.maximum.accumulate(np.clip(bounds, 0, n_items))
    return [(int(bounds[r]), int(bounds[r + 1])) for r in range(world)]


def local_items(off: np.ndarray, rank: int, world: int):
    """(item_begin, item_end, factor_begin, factor_end, local offsets) of a rank."""
    off = np.asarray(off, dtype=np.int64)
    i0, i1 = balanced_item_ranges(off, world)[rank]
    f0, f1 = int(off[i0]), int(off[i1])
    return i0, i1, f0, f1, (off[i0:i1 + 1] - f0).astype(np.int32)


def gather_items(J_local: torch.Tensor, ranges: list, group=None) -> torch.Tensor:
    """Assemble the full J from every rank's contiguous slice (all_gather of
    padded slices; the only exchange of the sharded Coulomb matrix)."""
    world = dist.get_world_size(group)
    longest = max(e - b for b, e in ranges)
    buf = torch.zeros(longest, dtype=J_local.dtype, device=J_local.device)
    buf[: J_local.numel()] = J_local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([parts[r][: e - b] for r, (b, e) in enumerate(ranges)])


def column_ranges(R_f: int, world: int) -> list:
    """Contiguous split of R_f factor columns for sharded convolutions."""
    edges = np.linspace(0, R_f, world + 1).round().astype(int)
    return [(int(edges[r]), int(edges[r + 1])) for r in range(world)]
