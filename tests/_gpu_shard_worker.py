"""One rank of the two-process sharded GPU build (run by
tests/test_gpu_shard.py, not collected by pytest).  The rank builds its
balanced shard of the small grid's clusters with libgale on cuda:0, takes
its global edge base from the gloo all-gather of per-rank edge counts, and
prints one JSON line with digests of its relation arrays."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch.distributed as dist  # noqa: E402

import gen  # noqa: E402
import paper_2507_15230_gb300 as gale  # noqa: E402
from paper_2507_15230_gb300 import shard  # noqa: E402


def main():
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=0) as ctx:
        I_V, I_T, _ = ctx.intervals()
        work = np.diff(I_T) + np.array([ctx.working_set(k)[0].size for k in range(ctx.K)])
        lo, hi = shard.shard_ranges(work, world)[rank]
        ctx.build(np.arange(lo, hi, dtype=np.int32), gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        out = ctx.export(gale.ALL)
    local_edges = int(out["et_w"].size)
    base, total = shard.edge_base(local_edges, dist)
    first, pos, firsts = 0, 0, []
    for k in range(lo, hi):
        nvk = int(I_V[k + 1] - I_V[k])
        firsts.append(base + first)
        first += int(out["et_uoff"][pos + nvk])
        pos += nvk + 1
    digests = {n: int(a.astype(np.int64).sum() * 1000003 + a.size) for n, a in out.items()}
    print(json.dumps({"rank": rank, "lo": int(lo), "hi": int(hi), "local_edges": local_edges, "base": base,
                      "total": total, "first_edges": firsts, "digests": digests}), flush=True)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
