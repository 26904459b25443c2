"""The critical-point classifier against fields whose critical points are
known, on oracle relations (no GPU)."""
import numpy as np

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
