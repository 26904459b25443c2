"""The oracle's per-cluster localized producer (working sets gathered once,
each cluster built from its own working set, threads over the clusters)
against the oracle's global definitions, which the closed forms, invariants
and brute force of test_oracle_pins.py pin: per-cluster sizes, a digest of
every cluster's ten arrays, and full arrays for sampled clusters."""
import numpy as np
import pytest

import gen
import oracle

KEYS = ("vt_off", "vt_val", "vv_off", "vv_val", "eu_off", "e_w", "et_off", "et_val", "tt_off", "tt_val")


@pytest.mark.parametrize("which", ["grid", "delaunay", "grid_uneven"])
def test_localized_equals_global(which):
    if which == "grid":
        m = gen.small_grid(with_field=False)
    elif which == "delaunay":
        m = gen.delaunay_mesh(3000, seed=18, kd_cap=256, with_field=False)
    else:
        m = gen.freudenthal_mesh(10, 40, seed=5, jitter=0.3, with_field=False)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    for threads in (1, 3):
        sizes, dig, sec = oracle.localized_build(canon, threads)
        assert np.array_equal(sizes, oracle.cluster_sizes(rel, canon))
        assert all(int(dig[k]) == oracle.relation_digest(oracle.cluster_view(rel, canon, k))
                   for k in range(m.nclusters))
        assert sec[0] >= 0 and sec[1] >= 0
    for k in (0, m.nclusters // 2, m.nclusters - 1):
        got, want = oracle.localized_cluster(canon, k), oracle.cluster_view(rel, canon, k)
        for n in KEYS:
            assert np.array_equal(got[n], want[n]), (k, n)


def test_digest_sees_a_planted_mistake():
    m = gen.small_grid(with_field=False)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    v = oracle.cluster_view(rel, canon, 3)
    d = oracle.relation_digest(v)
    for n in ("vt_val", "et_val", "tt_val", "e_w"):
        bad = dict(v)
        a = np.array(v[n]).copy()
        a[[0, 1]] = a[[1, 0]]  # two entries swapped
        bad[n] = a
        assert oracle.relation_digest(bad) != d, n
        bad[n] = np.concatenate([v[n], [0]])  # one entry too many
        assert oracle.relation_digest(bad) != d, n


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_localized_equals_global_on_non_manifold_soups(seed):
    """Random tet soups over a few vertices, with triangles in many tets:
    the localized producer's TT rows (from each cluster's working set and
    face halo) equal the global definition's."""
    rng = np.random.default_rng(900 + seed)
    nv, nt, K = int(rng.integers(8, 11)), int(rng.integers(40, 60)), int(rng.integers(2, 5))
    seen, tv = set(), []
    while len(tv) < nt:
        q = tuple(sorted(rng.choice(nv, 4, replace=False).tolist()))
        if q not in seen:
            seen.add(q)
            tv.append(list(rng.permutation(q)))
    seg = rng.integers(0, K, nv)
    seg[:K] = np.arange(K)
    rng.shuffle(seg)
    tv, seg = np.array(tv, np.int32), seg.astype(np.int32)
    canon, rel = oracle.build_all(nv, tv, seg, K)
    assert np.diff(rel["tt_off"]).max() > 4
    sizes, dig, _ = oracle.localized_build(canon, 2)
    assert np.array_equal(sizes, oracle.cluster_sizes(rel, canon))
    for k in range(K):
        assert int(dig[k]) == oracle.relation_digest(oracle.cluster_view(rel, canon, k))
        got, want = oracle.localized_cluster(canon, k), oracle.cluster_view(rel, canon, k)
        for n in KEYS:
            assert np.array_equal(got[n], want[n]), (k, n)
