"""Seed sharding of one PROPAGATE problem over ranks (torch.distributed).

Seeds never interact: bit i of every signature depends only on seed i (the
set signatures of Sec. 4). So one problem splits by seed words with no
per-round exchange. Each rank runs PROPAGATE-P on its own slice of the seeds
over a full replica of the graph, to its own fixpoint. The only exchange is
at the end: the ranks take the maximum of their round counts T, pad their
count rows to it, and all-gather the per-seed count columns. m_active is a
property of each rank's seed slice, so it is reported per rank, not summed
into the whole problem's.

    lo, hi = seed_shard(s, rank, world)
    res = propagate_p(G, seeds[lo:hi])
    counts = gather_counts(res.counts, world)   # (T+1, s) on every rank
"""
from __future__ import annotations

import numpy as np


def seed_shard(s: int, rank: int, world: int, word: int = 64) -> tuple[int, int]:
    """[lo, hi) of the seeds rank owns: whole 64-seed words, split as evenly
    as the words allow (ranks past the last word get an empty slice)."""
    if world < 1 or not 0 <= rank < world or s < 0:
        raise ValueError("bad shard arguments")
    words = -(-s // word)
    per, extra = divmod(words, world)
    w0 = rank * per + min(rank, extra)
    w1 = w0 + per + (1 if rank < extra else 0)
    return min(w0 * word, s), min(w1 * word, s)


def gather_counts(local: np.ndarray, world: int, group=None) -> np.ndarray:
    """All-gathers per-seed count columns (rows = rounds 0..T_local) from
    every rank, in rank order, padded with zero rows to the largest T."""
    import torch
    import torch.distributed as dist
    local = np.ascontiguousarray(local, dtype=np.uint32)
    if world == 1:
        return local
    rows = torch.tensor([local.shape[0], local.shape[1]], dtype=torch.int64)
    sizes = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, rows, group=group)
    T1 = int(max(int(x[0]) for x in sizes))
    widths = [int(x[1]) for x in sizes]
    wmax = max(widths)
    pad = np.zeros((T1, wmax), dtype=np.int64)  # int64: gloo has no uint32
    pad[:local.shape[0], :local.shape[1]] = local
    parts = [torch.zeros((T1, wmax), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(pad), group=group)
    cols = [p.numpy()[:, :w] for p, w in zip(parts, widths)]
    return np.concatenate(cols, axis=1).astype(np.uint32)
