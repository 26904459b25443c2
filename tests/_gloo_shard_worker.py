"""One rank of the two-process sharding test (run by tests/test_shard_gloo.py,
not collected by pytest).  Each rank takes its balanced shard of the small
grid's clusters, builds it with the oracle's per-cluster relations (the CPU
stand-in for its GPU), gets its global edge base from the all-gather, and
prints what it found as one JSON line."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch.distributed as dist  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402
from paper_2507_15230_gb300 import shard  # noqa: E402


def main():
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    m = gen.small_grid(with_field=False)
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    I_T = canon["I_T"]
    work = np.array([len(oracle.working_set(canon, k)[0]) + (I_T[k + 1] - I_T[k]) for k in range(m.nclusters)])
    lo, hi = shard.shard_ranges(work, world)[rank]
    local_edges = 0
    first_edges = []
    for k in range(lo, hi):
        r = oracle.cluster_relations(canon, k)
        first_edges.append(local_edges)
        local_edges += int(r["ne"])
    base, total = shard.edge_base(local_edges, dist)
    print(json.dumps({"rank": rank, "lo": int(lo), "hi": int(hi), "local_edges": local_edges, "base": base,
                      "total": total, "first_edges": [base + e for e in first_edges]}), flush=True)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
