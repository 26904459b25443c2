"""Sharding clusters across GPUs (one process per GPU).

Clusters are independent given their working sets (the internal tets, the
external tets T_ex and the face halo, Section 4.3), so the build shards with
no exchange of relations.  Each rank takes one contiguous range of cluster
ids, with the ranges balanced by working-set size, and builds it alone.  The
only quantity that crosses ranks is the number of owned edges per shard:
global edge ids (the paper's I_E, Section 4.3) are the edge's index within
its cluster plus the edges of all earlier clusters, so each rank needs the
exclusive prefix of the per-shard edge counts - one all-gather of one
integer per rank.
"""
from __future__ import annotations

import numpy as np


def shard_ranges(work: np.ndarray, world: int) -> list[tuple[int, int]]:
    """Split clusters 0..K-1 into `world` contiguous ranges [lo, hi) whose
    summed `work` (e.g. |T_k| + |halo_k| per cluster) is as even as a
    prefix split allows: the cut before rank r is the first cluster at which
    the running total reaches r/world of the whole.  Empty ranges are
    possible only when K < world."""
    work = np.asarray(work, dtype=np.float64)
    if work.ndim != 1:
        raise ValueError("work must be one value per cluster")
    if world < 1:
        raise ValueError("world must be >= 1")
    if (work < 0).any():
        raise ValueError("work must be non-negative")
    K = work.size
    csum = np.concatenate([[0.0], np.cumsum(work)])
    total = csum[-1]
    cuts = [0]
    for r in range(1, world):
        c = int(np.searchsorted(csum, total * r / world, side="left")) if total > 0 else (K * r) // world
        cuts.append(min(max(c, cuts[-1]), K))
    cuts.append(K)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def edge_base(local_edges: int, dist=None) -> tuple[int, int]:
    """Global id of this rank's first owned edge, and the total edge count:
    the exclusive scan of every rank's owned-edge count, in rank order
    (ranks hold consecutive cluster ranges).  `dist` is torch.distributed
    (None or not initialised: a single rank)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return 0, int(local_edges)
    import torch
    world, rank = dist.get_world_size(), dist.get_rank()
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    mine = torch.tensor([int(local_edges)], dtype=torch.int64, device=dev)
    allc = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(allc, mine)
    counts = [int(t.item()) for t in allc]
    return int(sum(counts[:rank])), int(sum(counts))
