"""Pins of the oracle's discrete gradient (Section 5.1, DiscreteGradient):
a hand-worked tetrahedron, Forman's conditions (each simplex critical or in
one facet pair, pairs inside one lower star, no closed V-path), the Euler
characteristic, a linear field on a convex mesh (one critical cell), and
the topology of every lower link (an optimal lower-star gradient has as many
critical cells as the lower link's reduced Betti numbers).  Planted mistakes
in the oracle's result must fail them."""
import json
import os

import numpy as np
import pytest

import gen
import oracle
from dg_util import critical_by_vertex, lower_link_prediction, violations

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def grid_case(n, K, seed, ties=5):
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=seed)
    nv = xyz.shape[0]
    seg = np.random.default_rng(seed).integers(0, K, nv).astype(np.int32)
    canon = oracle.canonicalize(nv, tv, seg, K)
    f = np.random.default_rng(seed + 9).integers(0, ties, nv).astype(np.float32)
    vp = np.asarray(canon["vperm"])
    return canon, f[vp].astype(np.float64), vp, xyz[vp]


def delaunay_case(npts, seed):
    m = gen.delaunay_mesh(npts, seed=seed, kd_cap=128, with_field=True)
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    vp = np.asarray(canon["vperm"])
    return canon, np.asarray(m.field, np.float32)[vp].astype(np.float64), vp


def test_single_tet_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "dg_single_tet.json")))
    canon = {"rows": np.array(g["rows"], np.int32), "nv": 4}
    r = oracle.lower_star_gradient(canon, g["field"], np.arange(4))
    assert [[list(a), list(b)] for a, b in r["pairs"]] == g["pairs"]
    assert [list(c) for c in r["critical"]] == g["critical"]


@pytest.mark.parametrize("n,K,seed,ties", [(2, 1, 0, 3), (3, 4, 1, 2), (4, 7, 2, 5), (4, 3, 3, 1000)])
def test_forman_conditions_euler_and_lower_links(n, K, seed, ties):
    canon, f, inid, _ = grid_case(n, K, seed, ties)
    r = oracle.lower_star_gradient(canon, f, inid)
    assert violations(canon["rows"], f, inid, r["pairs"], r["critical"]) == []
    pred = lower_link_prediction(canon["rows"], f, inid)
    assert critical_by_vertex(r["critical"], f, inid, int(canon["nv"])) == pred


def test_delaunay_lower_links():
    canon, f, inid = delaunay_case(400, seed=5)
    r = oracle.lower_star_gradient(canon, f, inid)
    assert violations(canon["rows"], f, inid, r["pairs"], r["critical"]) == []
    assert critical_by_vertex(r["critical"], f, inid, int(canon["nv"])) == lower_link_prediction(canon["rows"], f,
                                                                                                   inid)


def test_linear_field_has_one_critical_cell():
    canon, _, inid, xyz = grid_case(4, 5, 7)
    f = (xyz[:, 0] + 0.37 * xyz[:, 1] + 0.11 * xyz[:, 2]).astype(np.float32).astype(np.float64)
    r = oracle.lower_star_gradient(canon, f, inid)
    assert len(r["critical"]) == 1
    v = int(np.argmin(f))
    assert r["critical"] == [(v,)]


def test_constant_field_follows_input_ids():
    # all values tie: the order is the input id order, itself a valid field
    canon, _, inid, _ = grid_case(3, 2, 4)
    f = np.zeros(int(canon["nv"]))
    r = oracle.lower_star_gradient(canon, f, inid)
    assert violations(canon["rows"], f, inid, r["pairs"], r["critical"]) == []
    assert critical_by_vertex(r["critical"], f, inid, int(canon["nv"])) == lower_link_prediction(canon["rows"], f,
                                                                                                   inid)


def test_planted_mistakes_fail():
    canon, f, inid, _ = grid_case(3, 4, 11, 4)
    rows = canon["rows"]
    nv = int(canon["nv"])
    r = oracle.lower_star_gradient(canon, f, inid)
    pairs, crit = list(r["pairs"]), list(r["critical"])
    pred = lower_link_prediction(rows, f, inid)
    key = lambda v: (f[v], int(inid[v]))

    def fails(p, c):
        return violations(rows, f, inid, p, c) != [] or critical_by_vertex(c, f, inid, nv) != pred

    assert not fails(pairs, crit)
    # a pairing step skipped: both simplices left critical
    i = next(i for i, (a, b) in enumerate(pairs) if len(a) == 2)
    assert fails(pairs[:i] + pairs[i + 1:], crit + list(pairs[i]))
    # a pair reversed
    assert fails(pairs[:i] + [(pairs[i][1], pairs[i][0])] + pairs[i + 1:], crit)
    # a vertex paired with another of its lower edges than the one chosen
    for j, (a, b) in enumerate(pairs):
        if len(a) != 1:
            continue
        v = a[0]
        lower = sorted({tuple(sorted((v, int(w)))) for t in rows if v in t for w in t
                        if int(w) != v and key(int(w)) < key(v)} - {tuple(b)})
        if lower:
            assert fails(pairs[:j] + [(a, lower[0])] + pairs[j + 1:], crit)
            break
    else:
        pytest.fail("no vertex with a second lower edge")
    # a pair moved across lower stars: an edge paired with a triangle whose
    # highest vertex is another one
    for j, (a, b) in enumerate(pairs):
        if len(a) != 2:
            continue
        for t in rows:
            t = tuple(int(x) for x in t)
            if set(a) < set(t):
                for w in t:
                    c = tuple(sorted(set(a) | {w}))
                    if w not in a and max(c, key=key) != max(a, key=key):
                        assert fails(pairs[:j] + [(a, c)] + pairs[j + 1:], crit)
                        return
    pytest.fail("no cross-star triangle found")
