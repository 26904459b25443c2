"""The sharded build on the product: clusters split into balanced contiguous
shards (paper_2507_15230_gb300.shard), each shard built by libgale, must
give the single build's relations bit for bit, and the per-shard owned-edge
counts must turn into the global edge numbering (the paper's I_E, Section
4.3) through the exclusive scan that shard.edge_base computes.

One GPU: the shards are built one after the other in one process, and also
by two gloo ranks that share cuda:0 (their kernels never wait on each
other); the only exchange is the all-gather of one edge count per rank."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import gen
import oracle
import paper_2507_15230_gb300 as gale
from paper_2507_15230_gb300 import shard

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _work(ctx):
    I_V, I_T, sizes = ctx.intervals()
    ext = np.array([ctx.working_set(k)[0].size for k in range(ctx.K)])
    return np.diff(I_T) + ext


@pytest.mark.parametrize("which", ["grid", "delaunay"])
def test_sequential_shards_equal_single_build(which):
    m = gen.small_grid(with_field=False) if which == "grid" else gen.delaunay_mesh(6000, seed=9, kd_cap=256,
                                                                                    with_field=False)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    with gale.Context.load(m, device=0) as ctx:
        ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        whole = ctx.export(gale.ALL)
        for world in (2, 3):
            parts = []
            local_edges = []
            for lo, hi in shard.shard_ranges(_work(ctx), world):
                ids = np.arange(lo, hi, dtype=np.int32)
                ctx.build(ids, gale.ALL, gale.MODE_BATCHED)
                ctx.synchronize()
                parts.append(ctx.export(gale.ALL))
                local_edges.append(int(parts[-1]["et_w"].size))
            for name in whole:
                got = np.concatenate([p[name] for p in parts])
                assert np.array_equal(got, whole[name]), (world, name)
            # global edge ids: shard base (exclusive scan of the shard edge
            # counts) + the cluster's first edge within its shard
            bases = np.concatenate([[0], np.cumsum(local_edges)[:-1]])
            I_V = canon["I_V"]
            k = 0
            for (lo, hi), base, p in zip(shard.shard_ranges(_work(ctx), world), bases, parts):
                eu = p["et_uoff"]
                pos, first = 0, 0
                for kk in range(lo, hi):
                    nvk = int(I_V[kk + 1] - I_V[kk])
                    assert base + first == int(rel["eu_off"][I_V[kk]]), (world, kk)
                    first += int(eu[pos + nvk])
                    pos += nvk + 1
                    k += 1
            assert k == m.nclusters
            assert sum(local_edges) == int(rel["eu_off"][-1])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_build_their_shards_on_the_gpu():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "_gpu_shard_worker.py")], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=600)
        assert p.returncode == 0, err[-3000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    m = gen.small_grid(with_field=False)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    assert outs[0]["lo"] == 0 and outs[0]["hi"] == outs[1]["lo"] and outs[1]["hi"] == m.nclusters
    assert outs[1]["base"] == outs[0]["local_edges"]
    assert outs[0]["total"] == outs[1]["total"] == int(rel["eu_off"][-1])
    I_V = canon["I_V"]
    assert outs[0]["first_edges"] + outs[1]["first_edges"] == [int(rel["eu_off"][I_V[k]]) for k in range(m.nclusters)]
    # each rank's relations equal the oracle's for its clusters
    from parity_util import expected_bulk
    for o in outs:
        want = expected_bulk(rel, canon, range(o["lo"], o["hi"]))
        for name, digest in o["digests"].items():
            assert digest == int(np.asarray(want[name], np.int64).sum() * 1000003 + want[name].size), (o["rank"], name)
