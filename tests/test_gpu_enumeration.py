"""The sorted edge / triangle enumeration built on the GPU (a device context
with ET preconditioned) against the oracle: E, F, I_E, I_F and the boundary
relations looked up through it, on grids under random partitions, a
Delaunay mesh and a 400-tet star (the many-tets path of an edge)."""
import numpy as np
import pytest

import gen
import oracle
import paper_2507_15230_gb300 as gale

pytestmark = pytest.mark.gpu


def check(m):
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    want = oracle.enumerate_simplices(canon, "sorted")
    with gale.Context.load(m, device=0) as ctx:
        got = ctx.enumerate(gale.ENUM_SORTED)
        rows = ctx.rows()
        nF = got["F"].shape[0]
        fe = ctx.boundary(gale.REL_FE, np.arange(nF, dtype=np.int64))
        te = ctx.boundary(gale.REL_TE, np.arange(rows.shape[0], dtype=np.int64))
        tf = ctx.boundary(gale.REL_TF, np.arange(rows.shape[0], dtype=np.int64))
    assert [tuple(e) for e in got["E"].tolist()] == want["E"]
    assert [tuple(f) for f in got["F"].tolist()] == want["F"]
    assert got["I_E"].tolist() == want["I_E"] and got["I_F"].tolist() == want["I_F"]
    assert fe.tolist() == oracle.boundary(canon, want, "FE", range(nF))
    assert te.tolist() == oracle.boundary(canon, want, "TE", range(rows.shape[0]))
    assert tf.tolist() == oracle.boundary(canon, want, "TF", range(rows.shape[0]))


def test_small_grid():
    check(gen.small_grid(with_field=False))


@pytest.mark.parametrize("n,K,seed", [(3, 1, 0), (4, 9, 1), (6, 40, 2)])
def test_random_partitions(n, K, seed):
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=seed + 70)
    seg = np.random.default_rng(seed).integers(0, K, xyz.shape[0]).astype(np.int32)
    check(gen.Mesh(xyz, tv, seg, K))


def test_delaunay_and_high_degree_star():
    check(gen.delaunay_mesh(2000, seed=43, kd_cap=256, with_field=False))
    from test_gpu_parity import fan_mesh
    xyz, tv = fan_mesh()
    seg = np.random.default_rng(4).integers(0, 3, xyz.shape[0]).astype(np.int32)
    check(gen.Mesh(xyz, tv, seg, 3))


def test_first_appearance_stays_on_the_host_and_matches():
    m = gen.small_grid(with_field=False)
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    want = oracle.enumerate_simplices(canon, "first")
    with gale.Context.load(m, device=0) as ctx:
        got = ctx.enumerate(gale.ENUM_FIRST_APPEARANCE)
        again = ctx.enumerate(gale.ENUM_SORTED)  # then replaced by the device lists
    assert [tuple(e) for e in got["E"].tolist()] == want["E"]
    assert [tuple(f) for f in got["F"].tolist()] == want["F"]
    assert [tuple(e) for e in again["E"].tolist()] == sorted(want["E"])


def test_empty_clusters():
    """Cluster ids that own no vertex: empty intervals in I_E and I_F."""
    xyz, tv = gen.freudenthal_grid(4, permute=True, seed=77)
    seg = np.random.default_rng(3).choice(np.array([0, 2, 5, 7, 11], np.int32), xyz.shape[0]).astype(np.int32)
    m = gen.Mesh(xyz, tv, seg, 12)
    check(m)
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    want = oracle.coboundary(canon, oracle.enumerate_simplices(canon, "sorted"))
    with gale.Context.load(m, device=0) as ctx:
        ctx.enumerate(gale.ENUM_SORTED)
        got = ctx.coboundary()
    for name in ("VE", "VF", "EF", "FT"):
        off, val = got[name]
        assert val.tolist() == [x for r in want[name] for x in r], name


def test_device_lists_reach_the_host_in_any_query_order():
    """The sorted lists stay on the device until a query needs them: a
    boundary query first (the host copy and index), the lists after it
    (from the host copy), and the coboundary pass, which reuses the device
    copy; and the other order, with the lists straight from the device."""
    m = gen.small_grid(with_field=False)
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    want = oracle.enumerate_simplices(canon, "sorted")
    cbw = oracle.coboundary(canon, want)
    lib = gale.load_library()
    for boundary_first in (True, False):
        with gale.Context.load(m, device=0) as ctx:
            assert lib.gale_enumerate(ctx._h, gale.ENUM_SORTED) == 0
            nF = len(want["F"])
            if boundary_first:
                fe = ctx.boundary(gale.REL_FE, np.arange(nF, dtype=np.int64))
                got = ctx.enumeration()
                cb = ctx.coboundary()
            else:
                cb = ctx.coboundary()
                got = ctx.enumeration()
                fe = ctx.boundary(gale.REL_FE, np.arange(nF, dtype=np.int64))
            assert [tuple(e) for e in got["E"].tolist()] == want["E"]
            assert [tuple(f) for f in got["F"].tolist()] == want["F"]
            assert fe.tolist() == oracle.boundary(canon, want, "FE", range(nF))
            for name in ("VE", "VF", "EF", "FT"):
                assert cb[name][1].tolist() == [x for r in cbw[name] for x in r], name
