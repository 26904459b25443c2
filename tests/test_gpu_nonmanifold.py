"""Non-manifold meshes: a triangle shared by three or more tets.

TT(t) is every tet sharing exactly three vertices with t (Section 4.2), so a
tet on such a triangle has more than one partner across it.  A whole cluster
in shared memory or in global scratch finds those rows by a general pass over
its block; the results must equal the oracle's bit for bit, whatever the
mask, mode or cluster subset.  Clusters cut into parts assume a manifold
mesh, so a mesh whose cut clusters are not loads again uncut."""
import numpy as np
import pytest

import gen
import oracle
import paper_2507_15230_gb300 as gale
from parity_util import assert_bulk_equal, expected_bulk

pytestmark = pytest.mark.gpu

MASKS = (gale.ALL, gale.TT, gale.VT | gale.TT, gale.VV | gale.ET)


def _add_tets(m, faces, seg_new, seed):
    """m plus one new vertex and one new tet (face + vertex) per face; the
    new vertex sits just off the face's centroid."""
    rng = np.random.default_rng(seed)
    faces = np.asarray(faces, np.int32).reshape(-1, 3)
    c = m.xyz[faces].mean(axis=1) + rng.normal(0, 1e-3, (len(faces), 3)).astype(np.float32)
    nv = m.nv
    new_v = np.arange(nv, nv + len(faces), dtype=np.int32)
    tv_new = np.concatenate([faces, new_v[:, None]], axis=1)
    for row in tv_new:
        rng.shuffle(row)
    return gen.Mesh(np.concatenate([m.xyz, c.astype(np.float32)]), np.concatenate([m.tv, tv_new]).astype(np.int32),
                    np.concatenate([m.seg, np.asarray(seg_new, np.int32)]), m.nclusters, name=m.name + "+nm")


def _faces_of(tv):
    f = np.sort(tv[:, [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]], axis=2)
    return f  # [nt, 4, 3], face i opposite vertex i


def non_manifold_grid(n_extra=48, seed=3):
    """The 16^3 grid (kd leaves <= 64) with new tets on interior triangles:
    half on the face of a tet opposite its only vertex in the owning cluster
    (the face lies in the cluster's halo), half on random interior faces,
    every fourth triangle taking two new tets (four tets on one triangle).
    The new vertices go to the cluster of a face vertex or to a random one."""
    m = gen.small_grid(with_field=False)
    rng = np.random.default_rng(seed)
    tv, seg = m.tv, m.seg
    f = _faces_of(tv)
    flat = f.reshape(-1, 3)
    _, inv, cnt = np.unique(flat, axis=0, return_inverse=True, return_counts=True)
    interior = (cnt[inv.ravel()] == 2).reshape(-1, 4)
    s = seg[tv]  # [nt, 4]
    smin = s.min(axis=1)
    lone = (s == smin[:, None]).sum(axis=1) == 1
    opp = np.argmin(s, axis=1)
    halo_t = np.nonzero(lone & interior[np.arange(len(tv)), opp])[0]
    pick_h = rng.choice(halo_t, n_extra // 2, replace=False)
    faces = [f[t, opp[t]] for t in pick_h]
    cand = np.argwhere(interior)
    for t, i in cand[rng.choice(len(cand), n_extra - n_extra // 2, replace=False)]:
        faces.append(f[t, i])
    faces = np.unique(np.array(faces), axis=0)
    faces = np.concatenate([faces, faces[::4]])  # a second new tet on every fourth triangle
    seg_new = [seg[fc[rng.integers(3)]] if rng.random() < 0.5 else rng.integers(m.nclusters) for fc in faces]
    return _add_tets(m, faces, seg_new, seed)


def _check_all(ctx, m, canon, rel, seed):
    for mode in (gale.MODE_BATCHED, gale.MODE_PER_CLUSTER):
        ctx.build(None, gale.ALL, mode)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, np.arange(m.nclusters)))
    rng = np.random.default_rng(seed)
    ids = rng.permutation(m.nclusters)[: max(1, m.nclusters // 2)].astype(np.int32)
    for mask in MASKS:
        ctx.build(ids, mask, gale.MODE_BATCHED)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(mask), expected_bulk(rel, canon, ids, mask))


def test_three_tets_on_a_triangle():
    xyz = np.random.default_rng(0).random((6, 3)).astype(np.float32)
    tv = np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]], np.int32)
    seg = np.array([0, 0, 1, 1, 0, 1], np.int32)
    m = gen.Mesh(xyz, tv, seg, 2)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, 2)
    assert np.diff(rel["tt_off"]).tolist() == [2, 2, 2]
    with gale.Context.load(m, device=0) as ctx:
        _check_all(ctx, m, canon, rel, 0)


def _soup(rng, nv, nt, K):
    """Random tets over few vertices: many triangles in three or more tets."""
    seen, tv = set(), []
    while len(tv) < nt:
        q = tuple(sorted(rng.choice(nv, 4, replace=False).tolist()))
        if q not in seen:
            seen.add(q)
            tv.append(list(rng.permutation(q)))
    seg = rng.integers(0, K, nv)
    seg[:K] = np.arange(K)
    rng.shuffle(seg)
    return np.array(tv, np.int32), seg.astype(np.int32)


@pytest.mark.parametrize("i", range(6))
def test_random_soups(i):
    rng = np.random.default_rng(100 + i)
    nv = int(rng.integers(8, 16))
    tv, seg = _soup(rng, nv, int(rng.integers(30, 60)), int(rng.integers(1, 5)))
    K = int(seg.max()) + 1
    m = gen.Mesh(rng.random((nv, 3)).astype(np.float32), tv, seg, K)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, K)
    assert np.diff(rel["tt_off"]).max() > 4  # rows longer than a manifold allows
    with gale.Context.load(m, device=0) as ctx:
        _check_all(ctx, m, canon, rel, i)


_GRID = {}


def _grid():
    if not _GRID:
        m = non_manifold_grid()
        _GRID["m"] = m
        _GRID["ref"] = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    return _GRID["m"], _GRID["ref"]


def test_non_manifold_grid():
    m, (canon, rel) = _grid()
    assert np.diff(rel["tt_off"]).max() >= 5
    every = np.arange(m.nclusters, dtype=np.int32)
    with gale.Context.load(m, device=0) as ctx:
        # the marked clusters run from per-item bins; the hot kernel, which
        # lacks the general pass, would report them as an error instead
        assert any(b["per_item"] for b in ctx.bins())
        _check_all(ctx, m, canon, rel, 1)
        got = ctx.build_export(every, gale.ALL, chunks=3)
        assert_bulk_equal(got, expected_bulk(rel, canon, every))
        ctx.set_teams(64, 2)
        ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, every))
        ctx.set_teams(0, 0)
        ctx.autotune(gale.ALL, reps=1)
        ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, every))


@pytest.mark.parametrize("mode", ["loop", "batch"])
def test_non_manifold_served(mode):
    """Every cluster of the grid requested through the serving path (the
    device-resident loop, or a launch per batch) equals the oracle."""
    m, (canon, rel) = _grid()
    with gale.Context.load(m, device=0, cache_budget_bytes=64 << 20) as ctx:
        ctx.serve_configure(gale.SERVE_LOOP if mode == "loop" else gale.SERVE_BATCH)
        for k in range(ctx.K):
            for mask in (gale.ALL, gale.VT | gale.TT):
                v = ctx.request(k, mask, timeout_ns=20_000_000_000)
                got = gale.view_to_numpy(v)
                ctx.release(v)
                want = expected_bulk(rel, canon, [k], mask)
                for name, a in want.items():
                    assert np.array_equal(got[name], a), (k, mask, name)


def _spill_clusters(ctx):
    out, mem, at = [], ctx.bin_members(), 0
    for b in ctx.bins():
        if b["spill"]:
            out.extend(mem[at:at + b["clusters"]].tolist())
        at += b["clusters"]
    return np.array(sorted(c for c in out if c < ctx.K), np.int32)


def test_non_manifold_spill_clusters():
    """New tets on triangles inside clusters too large for shared memory:
    with cutting off, their global-scratch bins give the oracle's TT.  With
    the default cut those clusters would be cut into parts, which assume
    one partner per face: the load finds that in its counting pass and
    loads again with no cluster cut, with the same results."""
    base = gen.delaunay_mesh(60000, seed=11, with_field=False)
    with gale.Context.load(base, device=0, part_vertices=-1) as ctx:
        big = _spill_clusters(ctx)
    assert len(big) > 0
    rng = np.random.default_rng(7)
    s = base.seg[base.tv]
    inside = np.nonzero(np.isin(s, big).all(axis=1))[0]
    pick = rng.choice(inside, 24, replace=False)
    f = _faces_of(base.tv)
    faces = np.array([f[t, rng.integers(4)] for t in pick])
    m = _add_tets(base, faces, base.seg[faces[:, 0]], 8)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    assert np.diff(rel["tt_off"]).max() >= 5
    with gale.Context.load(m, device=0, part_vertices=-1) as ctx:
        assert any(b["spill"] for b in ctx.bins())
        _check_all(ctx, m, canon, rel, 2)
    with gale.Context.load(base, device=0) as ctx:
        assert ctx.info().nparts > 0  # the manifold mesh is cut
    with gale.Context.load(m, device=0) as ctx:
        assert ctx.info().nparts == 0 and any(b["spill"] for b in ctx.bins())
        _check_all(ctx, m, canon, rel, 3)


@pytest.mark.parametrize("order,oname", [(gale.ENUM_SORTED, "sorted"), (gale.ENUM_FIRST_APPEARANCE, "first")])
@pytest.mark.parametrize("pre", ["all", "no_tt"])
def test_non_manifold_coboundary(order, oname, pre):
    """VE, VF, EF and FT of non-manifold meshes equal the oracle's.  FT rows
    longer than two take the counted form: at once when the load's counting
    pass marked the mesh (TT preconditioned), else after the two-slot form
    overflows."""
    rng = np.random.default_rng(7)
    tv, seg = _soup(rng, 12, 50, 3)
    soup = gen.Mesh(rng.random((12, 3)).astype(np.float32), tv, seg, int(seg.max()) + 1)
    mask = gale.ALL if pre == "all" else gale.VT | gale.VV | gale.ET
    for m in (_grid()[0], soup):
        canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
        want = oracle.coboundary(canon, oracle.enumerate_simplices(canon, oname))
        assert max(len(r) for r in want["FT"]) >= 3
        with gale.Context.load(m, device=0, precondition_mask=mask) as ctx:
            ctx.enumerate(order)
            for which in (gale.CB_VE | gale.CB_VF | gale.CB_EF, gale.CB_FT, gale.CB_VE | gale.CB_FT):
                got = ctx.coboundary(which)
                for i, name in enumerate(("VE", "VF", "EF", "FT")):
                    if not which & (1 << i):
                        continue
                    off, val = got[name]
                    rows = want[name]
                    assert off.tolist() == np.concatenate([[0], np.cumsum([len(r) for r in rows])]).tolist(), name
                    assert val.tolist() == [x for r in rows for x in r], name


def test_non_manifold_noalloc():
    """The allocation-free build into caller-owned arrays runs the marked
    clusters from their per-item bins too, and equals the oracle."""
    import torch
    m, (canon, rel) = _grid()
    rng = np.random.default_rng(11)
    with gale.Context.load(m, device=0) as ctx:
        for ids in (np.arange(m.nclusters, dtype=np.int32), rng.permutation(m.nclusters)[:40].astype(np.int32)):
            want = expected_bulk(rel, canon, ids)
            out = {n: torch.full((max(int(a.size), 1),), -7, dtype=torch.int32, device="cuda") for n, a in want.items()}
            ctx.build_noalloc(ids, gale.ALL, out)
            got = {n: out[n][:a.size].cpu().numpy() for n, a in want.items()}
            assert_bulk_equal(got, want)
