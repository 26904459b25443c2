"""Sharding clusters across ranks (host logic, no GPU): balanced contiguous
shards, and the one exchange the sharded build needs - global edge ids from
an all-gather of per-shard edge counts - run as two gloo processes."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import gen
import oracle
from paper_2507_15230_gb300 import shard

HERE = os.path.dirname(os.path.abspath(__file__))


def test_shard_ranges_partition_and_balance():
    rng = np.random.default_rng(0)
    for K, world in [(1, 1), (7, 3), (100, 4), (65536, 8), (5, 8)]:
        work = rng.integers(1, 3000, size=K)
        r = shard.shard_ranges(work, world)
        assert len(r) == world and r[0][0] == 0 and r[-1][1] == K
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert all(lo <= hi for lo, hi in r)
        per = [work[lo:hi].sum() for lo, hi in r]
        # a prefix split is within one cluster's work of the even share
        assert max(per) <= work.sum() / world + work.max() + 1e-9
    assert shard.shard_ranges(np.zeros(6), 3) == [(0, 2), (2, 4), (4, 6)]
    with pytest.raises(ValueError):
        shard.shard_ranges(np.array([1.0, -1.0]), 2)


def test_edge_base_single_rank():
    assert shard.edge_base(17) == (0, 17)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_give_global_edge_ids():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "_gloo_shard_worker.py")], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    # shards cover the clusters in order; edge bases are the exclusive scan
    m = gen.small_grid(with_field=False)
    assert outs[0]["lo"] == 0 and outs[0]["hi"] == outs[1]["lo"] and outs[1]["hi"] == m.nclusters
    assert outs[0]["base"] == 0 and outs[1]["base"] == outs[0]["local_edges"]
    assert outs[0]["total"] == outs[1]["total"] == outs[0]["local_edges"] + outs[1]["local_edges"]
    # each cluster's first global edge id equals the global oracle's numbering
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    eu = rel["eu_off"]
    I_V = canon["I_V"]
    want = [int(eu[I_V[k]]) for k in range(m.nclusters)]
    got = outs[0]["first_edges"] + outs[1]["first_edges"]
    assert got == want
    assert outs[0]["total"] == int(eu[-1])
