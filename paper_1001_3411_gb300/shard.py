"""Spreading a batch of independent subvolumes over the ranks of a job.

Each rank runs its share as one batched pass (``Hop.hop_run_batch``); the
subvolumes are independent periodic problems, so no data crosses ranks and
no collective sits on the data path.  Shares are balanced by particle count
with the longest-processing-time rule: largest subvolume first, each to the
rank with the fewest particles so far (ties to the lower rank), which keeps
the largest share within one subvolume of the smallest.
"""
from __future__ import annotations

import numpy as np


def shard_subvolumes(sizes, world: int) -> list[list[int]]:
    """Subvolume indices of every rank (each list ascending)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    sizes = np.asarray(sizes, dtype=np.int64)
    order = sorted(range(len(sizes)), key=lambda b: (-int(sizes[b]), b))
    load = [0] * world
    share: list[list[int]] = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda q: (load[q], q))
        share[r].append(b)
        load[r] += int(sizes[b])
    return [sorted(s) for s in share]


def subset(pos, offsets, boxes, idx):
    """Positions, offsets and boxes of the subvolumes `idx` of a batch, in
    that order (positions copied into one contiguous array)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    boxes = np.asarray(boxes, dtype=np.float64)
    parts = [pos[offsets[b]:offsets[b + 1]] for b in idx]
    sizes = [offsets[b + 1] - offsets[b] for b in idx]
    sub_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    sub_pos = np.ascontiguousarray(np.concatenate(parts)) if parts else pos[:0]
    return sub_pos, sub_off, boxes[list(idx)]
