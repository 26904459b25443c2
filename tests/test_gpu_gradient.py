"""The discrete gradient (Section 5.1, DiscreteGradient) end to end: VE and
VF from the GPU coboundary pass, VT from the GPU cluster build, FE and TF
from the host boundary relations, the native consumer threads, compared
with the oracle - every pair on small meshes under both numberings, and on
sampled lower stars plus whole-mesh invariants on a 64^3 grid."""
import numpy as np
import pytest

import consumers
import gen
import oracle
import paper_2507_15230_gb300 as gale
from dg_util import pairs_from_ids

pytestmark = pytest.mark.gpu


def run(m, order):
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    f_c, inid = consumers.canonical_inputs(m.field, canon["vperm"])
    with gale.Context.load(m, device=0) as ctx:
        rel = consumers.gather_gradient_relations(ctx, order)
        g, _ = consumers.discrete_gradient(ctx, f_c, inid, rel=rel, nthreads=8)
        en = ctx.enumeration()
    return canon, f_c, inid, g, en


@pytest.mark.parametrize("order", [gale.ENUM_SORTED, gale.ENUM_FIRST_APPEARANCE])
def test_small_grid_every_pair(order):
    m = gen.small_grid()
    canon, f_c, inid, g, en = run(m, order)
    pairs, crit = pairs_from_ids(g, en["E"], en["F"], canon["rows"])
    want = oracle.lower_star_gradient(canon, f_c.astype(np.float64), inid)
    assert pairs == {(tuple(a), tuple(b)) for a, b in want["pairs"]}
    assert crit == {tuple(c) for c in want["critical"]}


def test_delaunay_every_pair():
    m = gen.delaunay_mesh(3000, seed=41, kd_cap=256, with_field=True)
    canon, f_c, inid, g, en = run(m, gale.ENUM_SORTED)
    pairs, crit = pairs_from_ids(g, en["E"], en["F"], canon["rows"])
    want = oracle.lower_star_gradient(canon, f_c.astype(np.float64), inid)
    assert pairs == {(tuple(a), tuple(b)) for a, b in want["pairs"]}
    assert crit == {tuple(c) for c in want["critical"]}


def test_grid64_sampled_lower_stars_and_euler():
    m = gen.freudenthal_mesh(64, 512, seed=3, field_seed=4, jitter=0.2, ngauss=16)
    canon, f_c, inid, g, en = run(m, gale.ENUM_SORTED)
    E, F, rows = en["E"], en["F"], canon["rows"]
    # up and down arrays mirror each other
    for up, down in (("v_up", "e_down"), ("e_up", "f_down"), ("f_up", "t_down")):
        u = np.asarray(g[up])
        i = np.nonzero(u >= 0)[0]
        assert np.array_equal(np.asarray(g[down])[u[i]], i)
        assert int((np.asarray(g[down]) >= 0).sum()) == i.size
    # Euler characteristic of the ball from the critical cells
    cv = int((g["v_up"] < 0).sum())
    ce = int(((g["e_down"] < 0) & (g["e_up"] < 0)).sum())
    cf = int(((g["f_down"] < 0) & (g["f_up"] < 0)).sum())
    ct = int((g["t_down"] < 0).sum())
    assert cv - ce + cf - ct == 1
    # sampled lower stars against the oracle, one by one
    rng = np.random.default_rng(5)
    sample = rng.choice(m.nv, 200, replace=False)
    sample = np.concatenate([sample, [int(np.argmax(f_c)), int(np.argmin(f_c))]])
    want = oracle.lower_star_gradient(canon, f_c.astype(np.float64), inid, vertices=sample)
    rank = np.empty(m.nv, np.int64)
    rank[np.lexsort((inid, f_c))] = np.arange(m.nv)
    in_s = np.zeros(m.nv, bool)
    in_s[sample] = True
    got_p, got_c = set(), set()
    tup = lambda a: tuple(int(x) for x in a)
    for v in sample:
        v = int(v)
        if g["v_up"][v] >= 0:
            got_p.add(((v,), tup(E[g["v_up"][v]])))
        else:
            got_c.add((v,))
    for simp, ups, downs, cof in ((E, "e_up", "e_down", F), (F, "f_up", "f_down", rows), (rows, None, "t_down", None)):
        top = np.asarray(simp)[np.arange(len(simp)), np.argmax(rank[np.asarray(simp)], axis=1)]
        for i in np.nonzero(in_s[top])[0]:
            up = g[ups][i] if ups else -1
            if up >= 0:
                got_p.add((tup(simp[i]), tup(cof[up])))
            elif g[downs][i] < 0:
                got_c.add(tup(simp[i]))
    assert got_p == {(tuple(a), tuple(b)) for a, b in want["pairs"]}
    assert got_c == {tuple(c) for c in want["critical"]}
