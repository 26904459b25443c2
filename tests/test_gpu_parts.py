"""Clusters cut into parts, against the CPU oracle bit for bit.

A cluster whose working set would not fit one CTA's shared memory is also
cut into parts: contiguous ranges of its own vertices, each built by its own
CTA straight into the cluster's output arrays (its offsets shifted by the
earlier parts', its TT rows placed at the cluster-level offsets the counting
pass found).  Batched builds (full, partial lists, the pipelined export)
build the parts; the per-cluster form, serving and the allocation-free build
keep building the whole cluster.  Small meshes force the cut with tiny part
sizes so that parts meet every case: parts of one or a few vertices, parts
whose faces need the halo, clusters of one part's size left whole."""
import numpy as np
import pytest

import gen
import oracle
import paper_2507_15230_gb300 as gale
from parity_util import assert_bulk_equal, expected_bulk

pytestmark = pytest.mark.gpu


def _mesh(kind):
    if kind == "grid":
        return gen.small_grid(with_field=False)
    return gen.delaunay_mesh(6000, seed=5, with_field=False)


_ORACLE = {}


def _oracle(kind, m):
    if kind not in _ORACLE:
        _ORACLE[kind] = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    return _ORACLE[kind]


@pytest.mark.parametrize("kind,pv", [("grid", 1), ("grid", 8), ("grid", 16), ("delaunay", 5), ("delaunay", 64)])
def test_cut_clusters_batched_equal_oracle(kind, pv):
    m = _mesh(kind)
    canon, rel = _oracle(kind, m)
    with gale.Context.load(m, device=0, part_vertices=pv, cut_bytes=1) as ctx:
        info = ctx.info()
        assert info.nparts > info.cut_clusters > 0
        bins = ctx.bins()
        assert any(b["parts"] > 0 for b in bins) and any(b["parts"] == -1 for b in bins), bins
        every = np.arange(m.nclusters)
        for _ in range(2):  # the second build replays the captured graph
            ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, every))
        rng = np.random.default_rng(pv)
        ids = rng.permutation(m.nclusters)[: max(2, m.nclusters // 3)].astype(np.int32)
        for mask in (gale.ALL, gale.VT | gale.TT, gale.ET, gale.VV):
            ctx.build(ids, mask, gale.MODE_BATCHED)
            ctx.synchronize()
            assert_bulk_equal(ctx.export(mask), expected_bulk(rel, canon, ids, mask))
        # the pipelined export: chunk boundaries fall between clusters, never
        # between the parts of one
        for chunks in (1, 3, 7):
            got = ctx.build_export(ids, gale.ALL, chunks=chunks)
            assert_bulk_equal(got, expected_bulk(rel, canon, ids))
        # the per-cluster form builds cut clusters whole
        ctx.build(ids[:20], gale.ALL, gale.MODE_PER_CLUSTER)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, ids[:20]))


def test_parts_after_autotune_and_views():
    kind = "delaunay"
    m = _mesh(kind)
    canon, rel = _oracle(kind, m)
    with gale.Context.load(m, device=0, part_vertices=32, cut_bytes=1) as ctx:
        ctx.autotune(gale.ALL, reps=1)
        ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, np.arange(m.nclusters)))
        # per-cluster views of a batched build of cut clusters
        cut = [k for b, s in zip(ctx.bins(), _bin_slices(ctx)) if b["parts"] == -1 for k in s]
        assert cut
        ids = np.array(sorted(cut)[:10], np.int32)
        ctx.build(ids, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        for i, k in enumerate(ids):
            got = gale.view_to_numpy(ctx.bulk_view(i))
            want = oracle.cluster_relations(canon, int(k))
            for g, w in [("vt_off", "vt_off"), ("vt_val", "vt_val"), ("vv_off", "vv_off"), ("vv_val", "vv_val"),
                         ("et_uoff", "eu_off"), ("et_w", "e_w"), ("et_off", "et_off"), ("et_val", "et_val"),
                         ("tt_off", "tt_off"), ("tt_val", "tt_val")]:
                assert np.array_equal(got[g].astype(np.int64), want[w].astype(np.int64)), (int(k), g)


def _bin_slices(ctx):
    members = ctx.bin_members()
    out, s = [], 0
    for b in ctx.bins():
        out.append([int(x) for x in members[s:s + b["clusters"]]])
        s += b["clusters"]
    return out


def test_no_cut_leaves_bins_unchanged():
    m = _mesh("grid")
    with gale.Context.load(m, device=0, part_vertices=-1, cut_bytes=1) as ctx:
        assert ctx.info().nparts == 0
        assert all(b["parts"] == 0 for b in ctx.bins())
        assert sorted(ctx.bin_members().tolist()) == list(range(m.nclusters))
