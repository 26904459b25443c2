"""Bit-exact parity of the CUDA producer with the CPU oracle, through the C
ABI.  Everything is integer indexing, so the tolerance is zero: every offset
and every id of every relation of every cluster must match."""
import numpy as np
import pytest

import gen
import oracle
import paper_2507_15230_gb300 as gale
from parity_util import assert_bulk_equal, expected_bulk

pytestmark = pytest.mark.gpu

MASKS = [gale.ALL, gale.VT, gale.VV, gale.ET, gale.TT, gale.VT | gale.VV | gale.TT, gale.VV | gale.ET]


@pytest.fixture(scope="module")
def small():
    m = gen.small_grid()
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    ctx = gale.Context.load(m, device=0)
    yield m, canon, rel, ctx
    ctx.close()


def test_sizes_match_oracle(small):
    m, canon, rel, ctx = small
    _, _, sizes = ctx.intervals()
    assert np.array_equal(sizes, oracle.cluster_sizes(rel, canon))


@pytest.mark.parametrize("mode", [gale.MODE_BATCHED, gale.MODE_PER_CLUSTER])
@pytest.mark.parametrize("mask", MASKS)
def test_small_all_clusters(small, mode, mask):
    m, canon, rel, ctx = small
    ctx.build(None, mask, mode)
    ctx.synchronize()
    got = ctx.export(mask)
    assert_bulk_equal(got, expected_bulk(rel, canon, range(m.nclusters), mask))


def test_small_subset_and_repeat(small):
    m, canon, rel, ctx = small
    rng = np.random.default_rng(3)
    ids = rng.permutation(m.nclusters)[:37]
    for mode in (gale.MODE_BATCHED, gale.MODE_PER_CLUSTER):
        ctx.build(ids, gale.ALL, mode)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, ids))
    # graph replay of the full build, twice, bit-identical
    ctx.build(None, gale.ALL, gale.MODE_BATCHED)
    ctx.synchronize()
    a = ctx.export(gale.ALL)
    ctx.build(None, gale.ALL, gale.MODE_BATCHED)
    ctx.synchronize()
    b = ctx.export(gale.ALL)
    for k in a:
        assert np.array_equal(a[k], b[k])
    assert_bulk_equal(a, expected_bulk(rel, canon, range(m.nclusters)))


@pytest.mark.parametrize("chunks", [0, 1, 3, 64])
@pytest.mark.parametrize("mask", [gale.ALL, gale.VV | gale.TT])
def test_build_export_pipelined(small, chunks, mask):
    """gale_build_export: chunked build with overlapping copies to host gives
    the oracle's arrays, for all clusters and for a shuffled subset, and
    leaves the same device bulk arrays as a plain batched build."""
    m, canon, rel, ctx = small
    got = ctx.build_export(None, mask, chunks=chunks)
    assert_bulk_equal(got, expected_bulk(rel, canon, range(m.nclusters), mask))
    assert_bulk_equal(ctx.export(mask), expected_bulk(rel, canon, range(m.nclusters), mask))
    ids = np.random.default_rng(5).permutation(m.nclusters)[:41]
    got = ctx.build_export(ids, mask, chunks=chunks)
    assert_bulk_equal(got, expected_bulk(rel, canon, ids, mask))


def test_views_match_oracle(small):
    m, canon, rel, ctx = small
    ctx.build(None, gale.ALL, gale.MODE_BATCHED)
    ctx.synchronize()
    for k in (0, 1, 63, m.nclusters - 1):
        v = ctx.bulk_view(k)
        got = gale.view_to_numpy(v)
        want = oracle.cluster_view(rel, canon, k)
        assert v.v_begin == canon["I_V"][k] and v.t_begin == canon["I_T"][k]
        for g, w in [("vt_off", "vt_off"), ("vt_val", "vt_val"), ("vv_val", "vv_val"), ("et_w", "e_w"),
                     ("et_val", "et_val"), ("tt_off", "tt_off"), ("tt_val", "tt_val")]:
            assert np.array_equal(got[g], want[w]), (k, g)


def partition_cases():
    cases = []
    for n, K, seed in [(3, 1, 0), (4, 1, 1), (5, 3, 2), (6, 40, 3), (8, 200, 4), (10, 17, 5)]:
        cases.append((n, K, seed))
    return cases


@pytest.mark.parametrize("case", partition_cases(), ids=lambda c: f"n{c[0]}-K{c[1]}")
def test_random_partitions(case):
    """Random segment ids (clusters that are not spatially compact, clusters
    owning no tets, one cluster for everything)."""
    n, K, seed = case
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=seed + 20)
    nv = xyz.shape[0]
    rng = np.random.default_rng(seed)
    seg = rng.integers(0, K, nv).astype(np.int32)
    m = gen.Mesh(xyz, tv, seg, K)
    canon, rel = oracle.build_all(nv, tv, seg, K)
    with gale.Context.load(m, device=0) as ctx:
        _, _, sizes = ctx.intervals()
        assert np.array_equal(sizes, oracle.cluster_sizes(rel, canon))
        for mode in (gale.MODE_BATCHED, gale.MODE_PER_CLUSTER):
            ctx.build(None, gale.ALL, mode)
            ctx.synchronize()
            assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, range(K)))


def test_empty_clusters_and_tiny_mesh():
    """Segments with no vertices, a segment with a single isolated vertex,
    a mesh of one tet."""
    tv = np.array([[0, 1, 2, 3]], np.int32)
    seg = np.array([0, 2, 2, 4, 4], np.int32)  # vertex 4 is isolated; clusters 1 and 3 empty
    m = gen.Mesh(None, tv, seg, 5)
    canon, rel = oracle.build_all(5, tv, seg, 5)
    with gale.Context.load(m, device=0) as ctx:
        for mode in (gale.MODE_BATCHED, gale.MODE_PER_CLUSTER):
            ctx.build(None, gale.ALL, mode)
            ctx.synchronize()
            assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, range(5)))


def test_paper_examples():
    """The worked examples of Sections 2.2 and 4.3 through the GPU path."""
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mesh_input_example.json")))
    tv, seg = np.array(g["tv"], np.int32), np.array(g["seg"], np.int32)
    m = gen.Mesh(None, tv, seg, g["nclusters"])
    with gale.Context.load(m, device=0) as ctx:
        _, _, sizes = ctx.intervals()
        assert [0] + np.cumsum(sizes[:, 2]).tolist() == g["expect"]["I_E"]
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "vv_two_tets.json")))
    tv, seg = np.array(g["tv"], np.int32), np.array(g["seg"], np.int32)
    m = gen.Mesh(None, tv, seg, 1)
    with gale.Context.load(m, device=0) as ctx:
        ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        out = ctx.export(gale.ALL)
        vp, _ = ctx.permutations()
        cid = np.argsort(vp)
        c0 = cid[0]
        vv = out["vv_val"][out["vv_off"][c0]:out["vv_off"][c0 + 1]]
        assert sorted(vp[vv].tolist()) == g["expect"]["VV"]["0"]


@pytest.mark.parametrize("npts,seed", [(20000, 5), (60000, 11)])
def test_delaunay_uneven_clusters(npts, seed):
    """Delaunay meshes of Gaussian-mixture points with uneven kd leaves of 32
    to 2,048 vertices: irregular stars and clusters too large for shared
    memory (their bins run in global scratch)."""
    m = gen.delaunay_mesh(npts, seed=seed, with_field=False)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    with gale.Context.load(m, device=0) as ctx:
        bins = ctx.bins()
        # members: every cluster, and the parts of the clusters cut for
        # batched builds
        assert sum(b["clusters"] for b in bins) == m.nclusters + ctx.info().nparts
        assert any(b["spill"] for b in bins), bins
        _, _, sizes = ctx.intervals()
        assert np.array_equal(sizes, oracle.cluster_sizes(rel, canon))
        for mode in (gale.MODE_BATCHED, gale.MODE_PER_CLUSTER):
            ctx.build(None, gale.ALL, mode)
            ctx.synchronize()
            assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, range(m.nclusters)))


@pytest.mark.parametrize("which", ["grid", "delaunay"])
def test_autotune_keeps_parity(which):
    """gale_autotune picks a block size and CTAs per SM per size bin by
    timing; the choice shows in the bins and the next full build (a fresh
    graph capture) is still bit-exact."""
    m = gen.small_grid() if which == "grid" else gen.delaunay_mesh(20000, seed=5, with_field=False)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    with gale.Context.load(m, device=0) as ctx:
        before = ctx.bins()
        best = ctx.autotune(gale.ALL, reps=1)
        after = ctx.bins()
        assert len(best) == len(before) == len(after)
        # bins of cut clusters are not timed (batched builds run their parts)
        assert all(ms > 0 for ms, b in zip(best, after) if b["parts"] != -1)
        for b0, b1 in zip(before, after):
            assert b1["clusters"] == b0["clusters"] and b1["spill"] == b0["spill"]
            assert b1["threads"] in (128, 256, 384, 512, 768, 1024)
            assert 1 <= b1["grid"] <= max(b0["clusters"], 1)
        for _ in range(2):
            ctx.build(None, gale.ALL, gale.MODE_BATCHED)
            ctx.synchronize()
            assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, range(m.nclusters)))


def test_contexts_do_not_shrink_each_others_launch_limits():
    """Kernel launch attributes are shared by every context of the process:
    loading a small mesh after one with large shared-memory plans must not
    stop the first one's large bins from launching."""
    big = gen.delaunay_mesh(60000, seed=11, with_field=False)
    canon, rel = oracle.build_all(big.nv, big.tv, big.seg, big.nclusters)
    with gale.Context.load(big, device=0) as c1:
        with gale.Context.load(gen.small_grid(with_field=False), device=0) as c2:
            for mode in (gale.MODE_BATCHED, gale.MODE_PER_CLUSTER):
                c1.build(None, gale.ALL, mode)
                c1.synchronize()
                assert_bulk_equal(c1.export(gale.ALL), expected_bulk(rel, canon, range(big.nclusters)))
                c2.build(None, gale.ALL, mode)
                c2.synchronize()


def fan_mesh(m_ring=200):
    """A vertex of degree 2 * m_ring: the centre of a ring of m_ring vertices
    between two poles, every tet (centre, pole, ring_i, ring_i+1).  Its VT
    row exceeds 256 entries and spans several 32-tet chunks."""
    ang = np.linspace(0, 2 * np.pi, m_ring, endpoint=False)
    xyz = np.zeros((m_ring + 3, 3), np.float32)
    xyz[1] = [0, 0, 1]
    xyz[2] = [0, 0, -1]
    xyz[3:, 0] = np.cos(ang)
    xyz[3:, 1] = np.sin(ang)
    tv = []
    for i in range(m_ring):
        a, b = 3 + i, 3 + (i + 1) % m_ring
        tv.append([0, 1, a, b])
        tv.append([0, 2, a, b])
    return xyz, np.array(tv, np.int32)


@pytest.mark.parametrize("K,seed", [(1, 0), (3, 1), (12, 2)])
def test_high_degree_vertex(K, seed):
    """A 400-tet star (16-bit star positions, masks of 13 32-tet chunks) under
    several partitions, every mask, both modes."""
    xyz, tv = fan_mesh()
    rng = np.random.default_rng(seed)
    perm = rng.permutation(xyz.shape[0]).astype(np.int32)
    tv = perm[tv]
    xyz = xyz[np.argsort(perm)]
    seg = rng.integers(0, K, xyz.shape[0]).astype(np.int32)
    seg[perm[0]] = 0
    m = gen.Mesh(xyz, tv, seg, K)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, K)
    with gale.Context.load(m, device=0) as ctx:
        _, _, sizes = ctx.intervals()
        assert np.array_equal(sizes, oracle.cluster_sizes(rel, canon))
        for mode in (gale.MODE_BATCHED, gale.MODE_PER_CLUSTER):
            for mask in (gale.ALL, gale.ET, gale.TT, gale.VV | gale.ET):
                ctx.build(None, mask, mode)
                ctx.synchronize()
                assert_bulk_equal(ctx.export(mask), expected_bulk(rel, canon, range(K), mask))


@pytest.mark.parametrize("mask", [gale.VT, gale.VV, gale.ET, gale.TT, gale.VT | gale.ET])
def test_spill_bins_every_mask(mask):
    """Clusters too large for shared memory under every relation mask,
    batched and one launch per cluster: with the default cut, batched builds
    run their parts and the per-cluster form their global-scratch bins; with
    cutting off, batched builds run the global-scratch bins too."""
    m = gen.delaunay_mesh(60000, seed=11, with_field=False)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    want = expected_bulk(rel, canon, range(m.nclusters), mask)
    for pv in (0, -1):
        with gale.Context.load(m, device=0, part_vertices=pv) as ctx:
            assert any(b["spill"] for b in ctx.bins())
            assert (ctx.info().nparts > 0) == (pv == 0)
            for mode in (gale.MODE_BATCHED, gale.MODE_PER_CLUSTER):
                ctx.build(None, mask, mode)
                ctx.synchronize()
                assert_bulk_equal(ctx.export(mask), want)


def test_more_than_255_upper_neighbours_is_rejected():
    """A vertex with more than 255 distinct upper neighbours (its edges'
    positions are kept in 8 bits) is rejected at load with EINVAL."""
    xyz, tv = fan_mesh(300)
    m = gen.Mesh(xyz, tv, np.zeros(xyz.shape[0], np.int32), 1)
    with pytest.raises(gale.GaleError) as ei:
        gale.Context.load(m, device=0)
    assert gale.STATUS[ei.value.status] == "EINVAL" and "255" in str(ei.value)
