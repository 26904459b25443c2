"""The critical-point classifier against fields whose critical points are
known, and the discrete-gradient consumer against the oracle, both on oracle
relations (no GPU)."""
import numpy as np
import pytest

import consumers
import gen
import oracle


def classify_all(m, f):
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    f_c, inid = consumers.canonical_inputs(f, canon["vperm"])
    out = np.empty(m.nv, np.int8)
    for k in range(m.nclusters):
        v = oracle.cluster_view(rel, canon, k)
        out[canon["I_V"][k]:canon["I_V"][k + 1]] = consumers.classify_cluster(
            f_c, inid, canon["rows"], canon["I_V"][k], v["vt_off"], v["vt_val"], v["vv_off"], v["vv_val"])
    xyz_c = m.xyz[canon["vperm"]]
    return out, xyz_c


def interior(xyz, n):
    return np.all((xyz > 0.5) & (xyz < n - 0.5), axis=1)


def test_linear_field_has_no_interior_critical_points():
    n = 8
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=4)
    seg, K = gen.kdtree_partition(xyz, 40)
    m = gen.Mesh(xyz, tv, seg, K)
    f = (xyz[:, 0] + 0.37 * xyz[:, 1] + 0.11 * xyz[:, 2]).astype(np.float32)
    cls, xyz_c = classify_all(m, f)
    assert np.all(cls[interior(xyz_c, n)] == -1)


def test_bowl_has_one_interior_minimum():
    n = 8
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=5)
    seg, K = gen.kdtree_partition(xyz, 40)
    m = gen.Mesh(xyz, tv, seg, K)
    c = np.array([3.6, 4.3, 3.9])
    f = ((xyz - c) ** 2).sum(1).astype(np.float32)
    cls, xyz_c = classify_all(m, f)
    inside = interior(xyz_c, n)
    assert (cls[inside] == 0).sum() == 1
    assert (cls[inside] == 3).sum() == 0
    # negated: one interior maximum
    cls2, _ = classify_all(m, -f)
    assert (cls2[inside] == 3).sum() == 1 and (cls2[inside] == 0).sum() == 0


# ---- discrete gradient consumer (Section 5.1) on oracle relations ----

def oracle_dg_relations(canon, order="sorted"):
    en = oracle.enumerate_simplices(canon, order)
    cb = oracle.coboundary(canon, en)
    rel = oracle.relations(canon)
    rows = canon["rows"]

    def csr(rs):
        return (np.concatenate([[0], np.cumsum([len(r) for r in rs])]).astype(np.int64),
                np.array([x for r in rs for x in r], np.int32))
    return en, dict(ve=csr(cb["VE"]), vf=csr(cb["VF"]), vt=(np.asarray(rel["vt_off"]), np.asarray(rel["vt_val"])),
                    ev=np.array(en["E"], np.int32).reshape(-1, 2), fv=np.array(en["F"], np.int32).reshape(-1, 3),
                    tv=rows)


def dg_matches_oracle(canon, f_c, inid, order="sorted", nthreads=4):
    from dg_util import pairs_from_ids
    en, rel = oracle_dg_relations(canon, order)
    g, _ = consumers.discrete_gradient_arrays(f_c, inid, **rel, nthreads=nthreads, grain=5)
    pairs, crit = pairs_from_ids(g, en["E"], en["F"], canon["rows"])
    want = oracle.lower_star_gradient(canon, f_c.astype(np.float64), inid)
    assert pairs == {(tuple(a), tuple(b)) for a, b in want["pairs"]}
    assert crit == {tuple(c) for c in want["critical"]}



@pytest.mark.parametrize("n,K,seed,ties,order", [(3, 1, 0, 3, "sorted"), (4, 6, 1, 4, "first"),
                                                 (5, 9, 2, 1000, "sorted")])
def test_dg_consumer_equals_oracle_on_grids(n, K, seed, ties, order):
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=seed + 30)
    seg = np.random.default_rng(seed).integers(0, K, xyz.shape[0]).astype(np.int32)
    canon = oracle.canonicalize(xyz.shape[0], tv, seg, K)
    f = np.random.default_rng(seed + 3).integers(0, ties, xyz.shape[0]).astype(np.float32)
    f_c, inid = consumers.canonical_inputs(f, canon["vperm"])
    dg_matches_oracle(canon, f_c, inid, order)


def test_dg_consumer_equals_oracle_on_delaunay_and_fan():
    m = gen.delaunay_mesh(500, seed=8, kd_cap=128, with_field=True)
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    f_c, inid = consumers.canonical_inputs(m.field, canon["vperm"])
    dg_matches_oracle(canon, f_c, inid)
    from test_gpu_parity import fan_mesh
    xyz, tv = fan_mesh(60)
    seg = np.zeros(xyz.shape[0], np.int32)
    canon = oracle.canonicalize(xyz.shape[0], tv, seg, 1)
    f = np.random.default_rng(2).normal(size=xyz.shape[0]).astype(np.float32)
    f[0] = 10.0  # the high-degree centre is the maximum: its lower star is its whole star
    f_c, inid = consumers.canonical_inputs(f, canon["vperm"])
    dg_matches_oracle(canon, f_c, inid)


@pytest.mark.parametrize("m_ring", [20, 22, 23, 29, 31])
@pytest.mark.parametrize("centre_top", [True, False])
def test_dg_consumer_lower_star_sizes_and_signed_zeros(m_ring, centre_top):
    """A fan centre with m_ring + 2 neighbours: its lower star spans the
    consumer's small-star orderings (22..33 lower edges when the centre is
    the maximum) and the general one.  Values repeat and include -0.0 next
    to +0.0, which are one value, so input ids break those ties."""
    from test_gpu_parity import fan_mesh
    xyz, tv = fan_mesh(m_ring)
    canon = oracle.canonicalize(xyz.shape[0], tv, np.zeros(xyz.shape[0], np.int32), 1)
    rng = np.random.default_rng(m_ring)
    f = rng.integers(-2, 3, xyz.shape[0]).astype(np.float32)
    f[rng.random(xyz.shape[0]) < 0.3] = -0.0
    f[rng.random(xyz.shape[0]) < 0.3] = 0.0
    if centre_top:
        f[0] = 10.0
    f_c, inid = consumers.canonical_inputs(f, canon["vperm"])
    dg_matches_oracle(canon, f_c, inid)


def test_dg_lower_stars_by_ranges_equal_the_threaded_run():
    """gale_dg_lower_stars over consecutive vertex ranges (keys computed on
    the fly) fills the same arrays as gale_dg_run (keys precomputed)."""
    xyz, tv = gen.freudenthal_grid(5, permute=True, seed=41)
    seg = np.random.default_rng(5).integers(0, 7, xyz.shape[0]).astype(np.int32)
    canon = oracle.canonicalize(xyz.shape[0], tv, seg, 7)
    f = np.random.default_rng(6).integers(-3, 4, xyz.shape[0]).astype(np.float32)
    f_c, inid = consumers.canonical_inputs(f, canon["vperm"])
    _, rel = oracle_dg_relations(canon)
    want, _ = consumers.discrete_gradient_arrays(f_c, inid, **rel, nthreads=3, grain=7)
    got = {k: np.full_like(v, -7) for k, v in want.items()}
    cuts = [0, 1, 50, 51, 130, len(f_c)]
    for b, e in zip(cuts[:-1], cuts[1:]):
        consumers.lower_stars_into(got, f_c, inid, b, e, **rel)
    for k in want:
        assert np.array_equal(got[k], want[k]), k


def test_dg_consumer_rejects_inconsistent_relations():
    xyz, tv = gen.freudenthal_grid(2, permute=True, seed=3)
    canon = oracle.canonicalize(xyz.shape[0], tv, np.zeros(xyz.shape[0], np.int32), 1)
    f_c, inid = consumers.canonical_inputs(np.arange(xyz.shape[0], dtype=np.float32), canon["vperm"])
    _, rel = oracle_dg_relations(canon)
    rel["ev"] = rel["ev"].copy()
    rel["ev"][:, :] = rel["ev"][::-1, :]  # edges no longer match their VE rows
    with pytest.raises(RuntimeError):
        consumers.discrete_gradient_arrays(f_c, inid, **rel, nthreads=2)


def test_csr_from_bulk_stitches_cluster_rows():
    """Per-cluster CSR pieces (offsets from 0 each) become one CSR over all
    vertices; the oracle's per-cluster VT rows give the global VT."""
    xyz, tv = gen.freudenthal_grid(3, permute=True, seed=5)
    K = 4
    seg = np.random.default_rng(2).integers(0, K, xyz.shape[0]).astype(np.int32)
    canon, rel = oracle.build_all(xyz.shape[0], tv, seg, K)
    offs, vals = [], []
    for k in range(K):
        v = oracle.cluster_view(rel, canon, k)
        offs.append(np.asarray(v["vt_off"], np.int32))
        vals.append(np.asarray(v["vt_val"], np.int32))
    off, val = consumers.csr_from_bulk(np.concatenate(offs), np.concatenate(vals), canon["I_V"])
    assert np.array_equal(off, np.asarray(rel["vt_off"], np.int64))
    assert np.array_equal(val, np.asarray(rel["vt_val"], np.int32))
