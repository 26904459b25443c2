"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, independent of the oracle's own code.

* closed forms of the Freudenthal subdivision (V, E, F, T, boundary faces,
  Euler characteristic, relation sizes, interior stars);
* brute force straight from the definitions (Section 2.2, Table 1; internal
  rule of Section 4.3) on tiny meshes, written without any of the oracle's
  derivations (no star-based shortcuts);
* the paper's worked examples (Section 2.2 Fig. relation-example; Section 4.3
  Fig. mesh-input with the interval array I_E of Section 4.4);
* invariants that hold for any mesh;
* planted mistakes in oracle output, which these checks must catch.
"""
import itertools
import json
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# brute force from the definitions
# ---------------------------------------------------------------------------

def brute_canon(nv, tv, seg):
    """Canonical numbering from the definitions: vertices ordered by
    (segment, input id); a tet is internal to the segment of its lowest
    canonical vertex, which is the smallest segment id among its vertices;
    tets ordered by (owner, input index)."""
    order = sorted(range(nv), key=lambda v: (seg[v], v))
    cid = {v: i for i, v in enumerate(order)}
    owner = [min(seg[v] for v in t) for t in tv]
    torder = sorted(range(len(tv)), key=lambda t: (owner[t], t))
    rows = [tuple(sorted(cid[v] for v in tv[t])) for t in torder]
    return order, cid, torder, rows, [owner[t] for t in torder]


def brute_relations(nv, rows):
    T = len(rows)
    sets = [set(r) for r in rows]
    VT = [[t for t in range(T) if v in sets[t]] for v in range(nv)]
    VV = [sorted({w for t in range(T) if v in sets[t] for w in sets[t] if w != v}) for v in range(nv)]
    edges = sorted({(u, w) for r in rows for u in r for w in r if u < w})
    ET = {e: [t for t in range(T) if e[0] in sets[t] and e[1] in sets[t]] for e in edges}
    TT = [[s for s in range(T) if s != t and len(sets[t] & sets[s]) == 3] for t in range(T)]
    return VT, VV, edges, ET, TT


def csr_rows(off, val):
    return [list(val[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


def matches_brute(rel, brute):
    """True iff the oracle's global result equals the brute-force one."""
    VT, VV, edges, ET, TT = brute
    if csr_rows(rel["vt_off"], rel["vt_val"]) != VT:
        return False
    if csr_rows(rel["vv_off"], rel["vv_val"]) != VV:
        return False
    got_edges = []
    for u in range(len(rel["eu_off"]) - 1):
        for e in range(rel["eu_off"][u], rel["eu_off"][u + 1]):
            got_edges.append((u, int(rel["e_w"][e])))
    if got_edges != edges:
        return False
    for i, e in enumerate(edges):
        if list(rel["et_val"][rel["et_off"][i]:rel["et_off"][i + 1]]) != ET[e]:
            return False
    return csr_rows(rel["tt_off"], rel["tt_val"]) == TT


def random_soup(rng, nv, nt, K):
    """Random tet soup: distinct 4-subsets of nv vertices (faces may be shared
    by more than two tets), random segment ids."""
    seen, tv = set(), []
    while len(tv) < nt:
        q = tuple(sorted(rng.choice(nv, 4, replace=False).tolist()))
        if q not in seen:
            seen.add(q)
            t = list(q)
            rng.shuffle(t)
            tv.append(t)
    seg = rng.integers(0, K, nv)
    seg[:K] = np.arange(K)  # every segment non-empty
    rng.shuffle(seg)
    return np.array(tv, np.int32), seg.astype(np.int32)


def tiny_cases():
    rng = np.random.default_rng(12345)
    cases = []
    for n in (1, 2, 3):
        xyz, tv = gen.freudenthal_grid(n, permute=True, seed=7 + n)
        nv = xyz.shape[0]
        for K in (1, 3, nv):
            seg = rng.integers(0, K, nv).astype(np.int32)
            cases.append((f"grid{n}-K{K}", nv, tv, seg, int(seg.max()) + 1))
    for i in range(4):
        nv = int(rng.integers(6, 14))
        tv, seg = random_soup(rng, nv, int(rng.integers(3, 25)), int(rng.integers(1, 4)))
        cases.append((f"soup{i}", nv, tv, seg, int(seg.max()) + 1))
    return cases


@pytest.mark.parametrize("case", tiny_cases(), ids=lambda c: c[0])
def test_brute_force_tiny(case):
    _, nv, tv, seg, K = case
    assert oracle.validate(nv, tv, seg, K) == oracle.OK
    canon = oracle.canonicalize(nv, tv, seg, K)
    order, cid, torder, rows, owners = brute_canon(nv, tv.tolist(), seg.tolist())
    assert canon["vperm"].tolist() == order
    assert canon["tperm"].tolist() == torder
    assert [tuple(r) for r in canon["rows"].tolist()] == rows
    assert np.array_equal(np.diff(canon["I_T"]), np.bincount(owners, minlength=K))
    assert np.array_equal(np.diff(canon["I_V"]), np.bincount(seg, minlength=K))
    rel = oracle.relations(canon)
    assert matches_brute(rel, brute_relations(nv, rows))


@pytest.mark.parametrize("case", tiny_cases(), ids=lambda c: c[0])
def test_per_cluster_equals_global(case):
    _, nv, tv, seg, K = case
    canon = oracle.canonicalize(nv, tv, seg, K)
    rel = oracle.relations(canon)
    for k in range(K):
        a = oracle.cluster_relations(canon, k)
        b = oracle.cluster_view(rel, canon, k)
        for key in ("vt_off", "vt_val", "vv_off", "vv_val", "eu_off", "e_w", "et_off", "et_val", "tt_off", "tt_val"):
            assert np.array_equal(a[key], b[key]), (k, key)


# ---------------------------------------------------------------------------
# closed forms of the Freudenthal grid
# ---------------------------------------------------------------------------

def freudenthal_counts(n):
    """V, E, F, T, boundary triangles of the n^3 Freudenthal grid, counted
    from the construction: axis edges 3n(n+1)^2, face diagonals 3n^2(n+1),
    one body diagonal per cube; triangles from Euler's formula for a ball
    (chi = 1); two boundary triangles per boundary square."""
    V = (n + 1) ** 3
    T = 6 * n ** 3
    E = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    F = 1 - V + E + T
    Fb = 6 * 2 * n * n
    return V, E, F, T, Fb


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8])
def test_freudenthal_closed_forms(n):
    V, E, F, T, Fb = freudenthal_counts(n)
    assert E == 7 * n ** 3 + 9 * n ** 2 + 3 * n
    assert F == 12 * n ** 3 + 6 * n ** 2
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=n)
    rng = np.random.default_rng(n)
    K = int(min(V, 1 + rng.integers(1, 20)))
    seg = rng.integers(0, K, V).astype(np.int32)
    K = int(seg.max()) + 1
    canon = oracle.canonicalize(V, tv, seg, K)
    rel = oracle.relations(canon)
    assert rel["vt_off"][-1] == 4 * T
    assert rel["vv_off"][-1] == 2 * E
    assert rel["ne"] == E
    assert rel["et_off"][-1] == 6 * T
    # every interior triangle lies in two tets, every boundary one in one
    assert rel["tt_off"][-1] == 2 * (F - Fb) == 4 * T - 12 * n * n
    # Euler characteristic of the ball from the oracle's own counts
    faces = {tuple(sorted(f)) for r in canon["rows"].tolist() for f in itertools.combinations(r, 3)}
    assert V - rel["ne"] + len(faces) - T == 1
    # interior vertices: 24 tets, 14 neighbours; interior edge multiplicities
    lattice = np.empty(V, np.int64)
    # recover lattice coordinates of canonical vertices from the unpermuted grid
    xyz0, _ = gen.freudenthal_grid(n, permute=False)
    coord = {tuple(p): i for i, p in enumerate(xyz0.astype(int).tolist())}
    for c in range(V):
        lattice[c] = coord[tuple(xyz[canon["vperm"][c]].astype(int).tolist())]
    ijk = np.stack([lattice % (n + 1), (lattice // (n + 1)) % (n + 1), lattice // (n + 1) ** 2], 1)
    interior = np.all((ijk > 0) & (ijk < n), axis=1)
    vt_deg = np.diff(rel["vt_off"])
    vv_deg = np.diff(rel["vv_off"])
    assert np.all(vt_deg[interior] == 24)
    assert np.all(vv_deg[interior] == 14)
    for u in range(V):
        for e in range(rel["eu_off"][u], rel["eu_off"][u + 1]):
            w = rel["e_w"][e]
            if not (interior[u] and interior[w]):
                continue
            d = np.abs(ijk[u] - ijk[w]).sum()
            mult = rel["et_off"][e + 1] - rel["et_off"][e]
            # axis edge 6, face diagonal 4, body diagonal 6
            assert mult == {1: 6, 2: 4, 3: 6}[int(d)], (u, w, d, mult)


def test_small_grid_sums(small_mesh):
    m = small_mesh
    V, E, F, T, Fb = freudenthal_counts(16)
    assert (m.nv, m.nt) == (4913, 24576)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    sizes = oracle.cluster_sizes(rel, canon)
    assert sizes[:, 0].sum() == 4 * T and sizes[:, 1].sum() == 2 * E and sizes[:, 2].sum() == E
    assert sizes[:, 3].sum() == 6 * T and sizes[:, 4].sum() == 4 * T - 12 * 16 * 16
    assert (E, F) == (31024, 50688)


# ---------------------------------------------------------------------------
# worked examples from the paper
# ---------------------------------------------------------------------------

def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_paper_vv_example():
    g = load_golden("vv_two_tets.json")
    tv, seg = np.array(g["tv"], np.int32), np.array(g["seg"], np.int32)
    canon = oracle.canonicalize(g["nv"], tv, seg, g["nclusters"])
    rel = oracle.relations(canon)
    inv = canon["vperm"]  # canonical -> input
    cid = canon["cid"]
    for v, want in g["expect"]["VV"].items():
        c = cid[int(v)]
        got = sorted(int(inv[w]) for w in rel["vv_val"][rel["vv_off"][c]:rel["vv_off"][c + 1]])
        assert got == want
    tinv = canon["tperm"]
    for t, want in g["expect"]["TT"].items():
        c = int(np.where(tinv == int(t))[0][0])
        got = sorted(int(tinv[s]) for s in rel["tt_val"][rel["tt_off"][c]:rel["tt_off"][c + 1]])
        assert got == want


def test_paper_mesh_input_example():
    g = load_golden("mesh_input_example.json")
    tv, seg = np.array(g["tv"], np.int32), np.array(g["seg"], np.int32)
    canon = oracle.canonicalize(g["nv"], tv, seg, g["nclusters"])
    rel = oracle.relations(canon)
    sizes = oracle.cluster_sizes(rel, canon)
    I_E = [0] + np.cumsum(sizes[:, 2]).tolist()
    assert I_E == g["expect"]["I_E"]
    # t1 internal to S1 (index 0), external to S2 (index 1)
    c = int(np.where(canon["tperm"] == 1)[0][0])
    owner = int(np.searchsorted(canon["I_T"], c, side="right") - 1)
    assert owner == g["expect"]["t1_owner"]
    ext, _ = oracle.working_set(canon, g["expect"]["t1_external_to"])
    assert c in ext.tolist()


# ---------------------------------------------------------------------------
# invariants on the small workload
# ---------------------------------------------------------------------------

def test_invariants_small(small_mesh):
    m = small_mesh
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    rows = canon["rows"]
    # TT symmetric; every face in at most two tets
    tt = csr_rows(rel["tt_off"], rel["tt_val"])
    for t, nb in enumerate(tt):
        assert len(nb) <= 4
        for s in nb:
            assert t in tt[s]
    # ET(u, w) = VT(u) intersect VT(w); VV(v) = union of VT(v)'s other vertices
    vt = csr_rows(rel["vt_off"], rel["vt_val"])
    rng = np.random.default_rng(0)
    for u in rng.choice(m.nv, 200, replace=False):
        nb = set()
        for t in vt[u]:
            nb |= set(rows[t].tolist())
        nb.discard(u)
        assert list(rel["vv_val"][rel["vv_off"][u]:rel["vv_off"][u + 1]]) == sorted(nb)
        for e in range(rel["eu_off"][u], rel["eu_off"][u + 1]):
            w = rel["e_w"][e]
            assert list(rel["et_val"][rel["et_off"][e]:rel["et_off"][e + 1]]) == sorted(set(vt[u]) & set(vt[w]))
    # clusters own contiguous vertex ranges and the tets of their lowest vertex
    owner_of_vertex = np.searchsorted(canon["I_V"], np.arange(m.nv), side="right") - 1
    assert np.array_equal(owner_of_vertex, m.seg[canon["vperm"]])
    t_owner = np.searchsorted(canon["I_T"], np.arange(m.nt), side="right") - 1
    assert np.array_equal(t_owner, owner_of_vertex[rows[:, 0]])
    assert np.all(np.diff(rows, axis=1) > 0)


def test_working_set_definition(small_mesh):
    m = small_mesh
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    rows = canon["rows"]
    for k in (0, 9, 64, m.nclusters - 1):
        v0, v1 = canon["I_V"][k], canon["I_V"][k + 1]
        t0, t1 = canon["I_T"][k], canon["I_T"][k + 1]
        touch = np.any((rows >= v0) & (rows < v1), axis=1)
        owned = np.zeros(m.nt, bool)
        owned[t0:t1] = True
        ext, halo = oracle.working_set(canon, k)
        assert ext.tolist() == np.where(touch & ~owned)[0].tolist()
        # every external tet is owned by an earlier cluster
        assert np.all(ext < t0)
        own_sets = [set(r) for r in rows[t0:t1].tolist()]
        want = [t for t in np.where(~touch)[0] if any(len(set(rows[t].tolist()) & s) == 3 for s in own_sets)]
        assert halo.tolist() == want


# ---------------------------------------------------------------------------
# input checks
# ---------------------------------------------------------------------------

def test_validation_rejects_bad_input():
    tv = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], np.int32)
    seg = np.array([0, 0, 1, 1, 1], np.int32)
    assert oracle.validate(5, tv, seg, 2) == oracle.OK
    assert oracle.validate(5, np.array([[0, 1, 2, 5]], np.int32), seg, 2) == oracle.EINVAL  # id out of range
    assert oracle.validate(5, np.array([[0, 1, 2, -1]], np.int32), seg, 2) == oracle.EINVAL
    assert oracle.validate(5, np.array([[0, 1, 1, 3]], np.int32), seg, 2) == oracle.EINVAL  # repeated vertex
    assert oracle.validate(5, np.array([[0, 1, 2, 3], [3, 2, 1, 0]], np.int32), seg, 2) == oracle.EINVAL  # duplicate
    assert oracle.validate(5, tv, np.array([0, 0, 2, 1, 1], np.int32), 2) == oracle.EINVAL  # segment out of range
    assert oracle.validate(5, tv, seg, 0) == oracle.EINVAL


def test_degenerate_partitions():
    """One cluster for everything, one vertex per cluster, empty clusters,
    clusters owning no tets."""
    xyz, tv = gen.freudenthal_grid(3, permute=True, seed=5)
    nv = xyz.shape[0]
    for seg, K in ((np.zeros(nv, np.int32), 1),
                   (np.arange(nv, dtype=np.int32), nv),
                   ((np.arange(nv) % 5 * 2).astype(np.int32), 11)):
        canon = oracle.canonicalize(nv, tv, seg, K)
        rel = oracle.relations(canon)
        order, cid, torder, rows, _ = brute_canon(nv, tv.tolist(), seg.tolist())
        assert matches_brute(rel, brute_relations(nv, rows))
        for k in range(K):
            a = oracle.cluster_relations(canon, k)
            b = oracle.cluster_view(rel, canon, k)
            assert all(np.array_equal(a[x], b[x]) for x in ("vt_val", "vv_val", "e_w", "et_val", "tt_val", "tt_off"))


# ---------------------------------------------------------------------------
# the checks above catch plausible mistakes
# ---------------------------------------------------------------------------

def _mutations(rel):
    """Copies of a correct result, each with one plausible mistake planted."""
    def cp():
        return {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in rel.items()}
    m = cp(); m["vv_val"] = np.delete(m["vv_val"], 3); m["vv_off"][2:] -= 1; yield "dropped VV entry", m
    m = cp(); v = m["vt_val"]; v[0], v[1] = v[1], v[0]; yield "VT row out of order", m
    m = cp(); m["et_val"][5] += 1; yield "ET value off by one", m
    m = cp(); m["e_w"][2] -= 1; yield "wrong edge endpoint", m
    m = cp(); m["tt_val"][0] = m["tt_val"][1]; yield "TT repeats a neighbour", m
    m = cp(); m["tt_off"][1] += 1; yield "TT offset shifted", m
    m = cp(); m["vt_val"] = m["vt_val"][::-1].copy(); yield "VT reversed", m


def test_pins_catch_planted_mistakes():
    xyz, tv = gen.freudenthal_grid(2, permute=True, seed=3)
    nv = xyz.shape[0]
    seg = (np.arange(nv) % 3).astype(np.int32)
    canon = oracle.canonicalize(nv, tv, seg, 3)
    rel = oracle.relations(canon)
    _, _, _, rows, _ = brute_canon(nv, tv.tolist(), seg.tolist())
    brute = brute_relations(nv, rows)
    assert matches_brute(rel, brute)
    for name, bad in _mutations(rel):
        assert not matches_brute(bad, brute), name


# ---------------------------------------------------------------------------
# edge / triangle enumeration and boundary relations (Sections 4.3, 4.4)
# ---------------------------------------------------------------------------

def test_enumeration_paper_example():
    """The worked example: I_E = [0, 9, 12], the triangle f5 = (v0, v3, v4)
    and FE(f5) = {e2, e6, e9} under first-appearance numbering; sorted
    numbering keeps I_E and the triangle sets but gives (v0, v4) the id e3."""
    g = load_golden("mesh_input_example.json")
    tv, seg = np.array(g["tv"], np.int32), np.array(g["seg"], np.int32)
    canon = oracle.canonicalize(g["nv"], tv, seg, g["nclusters"])
    first = oracle.enumerate_simplices(canon, "first")
    assert first["I_E"] == g["expect"]["I_E"]
    assert list(first["F"][5]) == g["expect"]["f5"]
    assert oracle.boundary(canon, first, "FE", [5]) == [g["expect"]["FE_f5"]]
    srt = oracle.enumerate_simplices(canon, "sorted")
    assert srt["I_E"] == g["expect"]["I_E"]
    f5 = srt["F"].index(tuple(g["expect"]["f5"]))
    assert oracle.boundary(canon, srt, "FE", [f5]) == [[2, 3, 9]]


@pytest.mark.parametrize("n,K,seed", [(1, 1, 0), (2, 3, 1), (3, 5, 2), (4, 9, 3)])
def test_enumeration_closed_forms_and_invariants(n, K, seed):
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=seed + 40)
    seg = np.random.default_rng(seed).integers(0, K, xyz.shape[0]).astype(np.int32)
    canon = oracle.canonicalize(xyz.shape[0], tv, seg, K)
    rows = canon["rows"]
    I_V = np.asarray(canon["I_V"])
    all_e = {(int(r[i]), int(r[j])) for r in rows for i in range(4) for j in range(i + 1, 4)}
    all_f = {(int(r[i]), int(r[j]), int(r[k])) for r in rows for i in range(4) for j in range(i + 1, 4)
             for k in range(j + 1, 4)}
    enums = {o: oracle.enumerate_simplices(canon, o) for o in ("sorted", "first")}
    for o, en in enums.items():
        E, F = en["E"], en["F"]
        assert len(E) == 7 * n ** 3 + 9 * n ** 2 + 3 * n == len(all_e) and set(E) == all_e
        assert len(F) == 12 * n ** 3 + 6 * n ** 2 == len(all_f) and set(F) == all_f
        for k in range(K):  # ownership by the lowest vertex
            for e in E[en["I_E"][k]:en["I_E"][k + 1]]:
                assert I_V[k] <= e[0] < I_V[k + 1]
            for f in F[en["I_F"][k]:en["I_F"][k + 1]]:
                assert I_V[k] <= f[0] < I_V[k + 1]
        te = oracle.boundary(canon, en, "TE", range(rows.shape[0]))
        tf = oracle.boundary(canon, en, "TF", range(rows.shape[0]))
        for t in range(rows.shape[0]):
            r = set(int(x) for x in rows[t])
            assert len(set(te[t])) == 6 and all(set(E[i]) <= r for i in te[t])
            assert len(set(tf[t])) == 4 and all(set(F[i]) <= r for i in tf[t])
            for fe in oracle.boundary(canon, en, "FE", tf[t]):  # a face's edges are edges of the tet
                assert set(fe) <= set(te[t])
    # the two numberings list the same simplices per segment; sorted is lexicographic
    s, f = enums["sorted"], enums["first"]
    assert s["I_E"] == f["I_E"] and s["I_F"] == f["I_F"]
    for k in range(K):
        a, b = s["I_E"][k], s["I_E"][k + 1]
        assert s["E"][a:b] == sorted(f["E"][a:b])
        a, b = s["I_F"][k], s["I_F"][k + 1]
        assert s["F"][a:b] == sorted(f["F"][a:b])


def enumeration_violations(canon, n, E, F, TE, FE):
    """The closed-form and structural checks above, as a list of failures."""
    rows = canon["rows"]
    bad = []
    if len(E) != 7 * n ** 3 + 9 * n ** 2 + 3 * n or len(set(E)) != len(E):
        bad.append("edge count")
    if len(F) != 12 * n ** 3 + 6 * n ** 2 or len(set(F)) != len(F):
        bad.append("triangle count")
    for t, te in enumerate(TE):
        r = set(int(x) for x in rows[t])
        if len(set(te)) != 6 or not all(0 <= i < len(E) and set(E[i]) <= r for i in te):
            bad.append(f"TE({t})")
            break
    for f, fe in enumerate(FE):
        if f >= len(F) or len(set(fe)) != 3 or not all(0 <= i < len(E) and set(E[i]) <= set(F[f]) for i in fe):
            bad.append(f"FE({f})")
            break
    return bad


def test_enumeration_planted_mistakes_fail():
    """The checks catch a dropped edge, a repeated triangle, a tetrahedron's
    edge list with a repeated pair, and FE ids off by one."""
    n = 2
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=7)
    seg = np.random.default_rng(3).integers(0, 3, xyz.shape[0]).astype(np.int32)
    canon = oracle.canonicalize(xyz.shape[0], tv, seg, 3)
    en = oracle.enumerate_simplices(canon, "first")
    E, F = en["E"], en["F"]
    TE = oracle.boundary(canon, en, "TE", range(canon["rows"].shape[0]))
    FE = oracle.boundary(canon, en, "FE", range(len(F)))
    assert enumeration_violations(canon, n, E, F, TE, FE) == []
    assert enumeration_violations(canon, n, E[:-1], F, TE, FE)  # dropped edge
    assert enumeration_violations(canon, n, E, F[:-1] + [F[0]], TE, FE)  # repeated triangle
    te_bad = [list(x) for x in TE]
    te_bad[0][5] = te_bad[0][4]  # a pair listed twice
    assert enumeration_violations(canon, n, E, F, te_bad, FE)
    fe_bad = [[(i + 1) % len(E) for i in x] for x in FE]  # ids off by one
    assert enumeration_violations(canon, n, E, F, TE, fe_bad)


@pytest.mark.parametrize("order", ["sorted", "first"])
@pytest.mark.parametrize("n,K,seed", [(1, 1, 0), (2, 3, 1), (3, 7, 2)])
def test_coboundary_closed_forms_and_transposes(order, n, K, seed):
    """VE, VF, EF, FT: totals 2E, 3F, 3F, 2F - F_boundary (F_boundary =
    12 n^2); interior vertices have 14 edges and 36 triangles; each is the
    transpose of a boundary relation (EV, FV, FE, TF - the last two pinned by
    the worked example); rows ascending."""
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=seed + 80)
    seg = np.random.default_rng(seed).integers(0, K, xyz.shape[0]).astype(np.int32)
    canon = oracle.canonicalize(xyz.shape[0], tv, seg, K)
    en = oracle.enumerate_simplices(canon, order)
    cb = oracle.coboundary(canon, en)
    E, F = en["E"], en["F"]
    nE, nF, nT = len(E), len(F), canon["rows"].shape[0]
    assert sum(map(len, cb["VE"])) == 2 * nE
    assert sum(map(len, cb["VF"])) == 3 * nF
    assert sum(map(len, cb["EF"])) == 3 * nF
    assert sum(map(len, cb["FT"])) == 2 * nF - 12 * n * n
    for key in cb:
        assert all(r == sorted(set(r)) for r in cb[key])
    # transposes
    fe = oracle.boundary(canon, en, "FE", range(nF))
    tf = oracle.boundary(canon, en, "TF", range(nT))
    assert sorted((e, f) for f, row in enumerate(fe) for e in row) == \
        sorted((e, f) for e, row in enumerate(cb["EF"]) for f in row)
    assert sorted((f, t) for t, row in enumerate(tf) for f in row) == \
        sorted((f, t) for f, row in enumerate(cb["FT"]) for t in row)
    assert sorted((v, i) for i, e in enumerate(E) for v in e) == \
        sorted((v, i) for v, row in enumerate(cb["VE"]) for i in row)
    assert sorted((v, i) for i, f in enumerate(F) for v in f) == \
        sorted((v, i) for v, row in enumerate(cb["VF"]) for i in row)
    if n >= 3:  # an interior vertex of the grid: the lattice point nearest the centre
        mid = int(np.argmin(np.abs(xyz - xyz.mean(axis=0)).sum(axis=1)))
        v = int(canon["cid"][mid])
        assert len(cb["VE"][v]) == 14 and len(cb["VF"][v]) == 36


@pytest.mark.parametrize("order", ["sorted", "first"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_coboundary_brute_force_soups(order, seed):
    """On random tet soups over a few vertices (triangles in up to a dozen
    tets: non-manifold), the enumeration holds exactly the vertex pairs and
    triples of the tets, and VE, VF, EF, FT equal containment tests over
    every simplex, written without the oracle's code."""
    from itertools import combinations
    rng = np.random.default_rng(500 + seed)
    nv = int(rng.integers(8, 13))
    tv, seg = random_soup(rng, nv, int(rng.integers(20, 60)), int(rng.integers(1, 4)))
    K = int(seg.max()) + 1
    canon = oracle.canonicalize(nv, tv, seg, K)
    en = oracle.enumerate_simplices(canon, order)
    cb = oracle.coboundary(canon, en)
    rows = [tuple(r) for r in canon["rows"].tolist()]
    E = [tuple(e) for e in en["E"]]
    F = [tuple(f) for f in en["F"]]
    assert sorted(E) == sorted({p for r in rows for p in combinations(r, 2)})
    assert sorted(F) == sorted({q for r in rows for q in combinations(r, 3)})
    assert cb["VE"] == [[i for i, e in enumerate(E) if v in e] for v in range(nv)]
    assert cb["VF"] == [[i for i, f in enumerate(F) if v in f] for v in range(nv)]
    assert cb["EF"] == [[i for i, f in enumerate(F) if set(e) <= set(f)] for e in E]
    assert cb["FT"] == [[t for t, r in enumerate(rows) if set(f) <= set(r)] for f in F]
    assert max(len(r) for r in cb["FT"]) >= 3
