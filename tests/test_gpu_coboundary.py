"""Coboundary relations VE, VF, EF, FT on the GPU (gale_build_coboundary),
in the ids of the edge / triangle enumeration, against the oracle, bit for
bit: the small grid under both numberings, random partitions, a 400-tet
star and a Delaunay mesh."""
import numpy as np
import pytest

import gen
import oracle
import paper_2507_15230_gb300 as gale

pytestmark = pytest.mark.gpu

ORDERS = [(gale.ENUM_SORTED, "sorted"), (gale.ENUM_FIRST_APPEARANCE, "first")]


def check(m, order, oname, which=gale.CB_VE | gale.CB_VF | gale.CB_EF | gale.CB_FT):
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    en = oracle.enumerate_simplices(canon, oname)
    want = oracle.coboundary(canon, en)
    with gale.Context.load(m, device=0) as ctx:
        ctx.enumerate(order)
        got = ctx.coboundary(which)
        for i, name in enumerate(("VE", "VF", "EF", "FT")):
            if not which & (1 << i):
                assert name not in got
                continue
            off, val = got[name]
            rows = want[name]
            assert off.size == len(rows) + 1, name
            assert off.tolist() == np.concatenate([[0], np.cumsum([len(r) for r in rows])]).tolist(), name
            assert val.tolist() == [x for r in rows for x in r], name


@pytest.mark.parametrize("order,oname", ORDERS)
def test_small_grid(order, oname):
    check(gen.small_grid(with_field=False), order, oname)


@pytest.mark.parametrize("n,K,seed", [(3, 1, 0), (4, 7, 1), (5, 30, 2)])
def test_random_partitions(n, K, seed):
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=seed + 90)
    seg = np.random.default_rng(seed).integers(0, K, xyz.shape[0]).astype(np.int32)
    for order, oname in ORDERS:
        check(gen.Mesh(xyz, tv, seg, K), order, oname)


def test_high_degree_star_and_subsets():
    from test_gpu_parity import fan_mesh
    xyz, tv = fan_mesh()
    seg = np.random.default_rng(4).integers(0, 3, xyz.shape[0]).astype(np.int32)
    m = gen.Mesh(xyz, tv, seg, 3)
    check(m, gale.ENUM_FIRST_APPEARANCE, "first")
    check(m, gale.ENUM_SORTED, "sorted", which=gale.CB_VF | gale.CB_FT)


def test_delaunay():
    check(gen.delaunay_mesh(3000, seed=41, kd_cap=256, with_field=False), gale.ENUM_SORTED, "sorted")


def test_errors():
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=0) as ctx:
        with pytest.raises(gale.GaleError) as ei:
            ctx.coboundary()
        assert gale.STATUS[ei.value.status] == "ENOTFOUND"
        ctx.enumerate(gale.ENUM_SORTED)
        with pytest.raises(gale.GaleError):
            ctx.coboundary(16)


@pytest.mark.parametrize("pre", [gale.TT, gale.VT | gale.VV, gale.ET])
def test_any_precondition_mask(pre):
    """The pass reads only the enumeration and the tet rows: it works
    whatever the context is preconditioned for (the sorted enumeration is
    built on the device with ET, on the host without)."""
    m = gen.small_grid(with_field=False)
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    want = oracle.coboundary(canon, oracle.enumerate_simplices(canon, "sorted"))
    with gale.Context.load(m, device=0, precondition_mask=pre) as ctx:
        ctx.enumerate(gale.ENUM_SORTED)
        got = ctx.coboundary()
    for name in ("VE", "VF", "EF", "FT"):
        off, val = got[name]
        assert val.tolist() == [x for r in want[name] for x in r], name


def test_enumeration_replaced_between_calls():
    """A new enumeration (another numbering) replaces the lookup structure."""
    m = gen.small_grid(with_field=False)
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    with gale.Context.load(m, device=0) as ctx:
        for order, oname in ORDERS + ORDERS[::-1]:
            ctx.enumerate(order)
            ctx.enumerate(order)  # twice: the earlier enumeration's memory may be reused
            got = ctx.coboundary(gale.CB_VE | gale.CB_EF)
            want = oracle.coboundary(canon, oracle.enumerate_simplices(canon, oname))
            for name in ("VE", "EF"):
                off, val = got[name]
                assert val.tolist() == [x for r in want[name] for x in r], (oname, name)


def transpose(idx, width, nrows):
    """CSR (offsets, values) of the relation whose row r lists the ids i
    with r among idx[i] (idx: int array [n, width]), rows sorted."""
    idx = np.asarray(idx, dtype=np.int64).reshape(-1, width)
    rows = idx.reshape(-1)
    vals = np.repeat(np.arange(idx.shape[0], dtype=np.int64), width)
    order = np.argsort(rows * np.int64(idx.shape[0]) + vals, kind="stable")
    off = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=nrows))])
    return off, vals[order]


@pytest.mark.parametrize("order", [gale.ENUM_SORTED, gale.ENUM_FIRST_APPEARANCE])
def test_full_size_transposes_of_boundary_relations(order):
    """At 128^3 (12.6M tets), every row of VE, VF, EF and FT equals the
    transpose of EV, FV (the enumeration), FE and TF (the host boundary
    lookups), and the totals match the Freudenthal closed forms."""
    n = 128
    m = gen.freudenthal_mesh(n, 512, seed=3, field_seed=4, jitter=0.3, with_field=False)
    with gale.Context.load(m, device=0) as ctx:
        en = ctx.enumerate(order)
        E, F = en["E"], en["F"]
        nE, nF = E.shape[0], F.shape[0]
        assert nE == 7 * n ** 3 + 9 * n ** 2 + 3 * n and nF == 12 * n ** 3 + 6 * n ** 2
        cb = ctx.coboundary()
        rows = ctx.rows()
        fe = ctx.boundary(gale.REL_FE, np.arange(nF, dtype=np.int64))
        tf = ctx.boundary(gale.REL_TF, np.arange(rows.shape[0], dtype=np.int64))
    want = {"VE": transpose(E, 2, m.nv), "VF": transpose(F, 3, m.nv), "EF": transpose(fe, 3, nE),
            "FT": transpose(tf, 4, nF)}
    totals = {"VE": 2 * nE, "VF": 3 * nF, "EF": 3 * nF, "FT": 4 * rows.shape[0]}
    for name, (off, val) in want.items():
        g_off, g_val = cb[name]
        assert g_val.size == totals[name], name
        assert np.array_equal(g_off, off), name
        assert np.array_equal(g_val, val), name
