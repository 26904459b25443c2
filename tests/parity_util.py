"""Expected bulk arrays from oracle results, in the product's layout:
clusters consecutive in list order, every offset array relative to its
cluster."""
import numpy as np

import oracle

KEYS = [("vt_off", "vt_off"), ("vt_val", "vt_val"), ("vv_off", "vv_off"), ("vv_val", "vv_val"),
        ("et_uoff", "eu_off"), ("et_w", "e_w"), ("et_off", "et_off"), ("et_val", "et_val"),
        ("tt_off", "tt_off"), ("tt_val", "tt_val")]
REL = {"vt_off": 1, "vt_val": 1, "vv_off": 2, "vv_val": 2, "et_uoff": 4, "et_w": 4, "et_off": 4, "et_val": 4,
       "tt_off": 8, "tt_val": 8}


def expected_bulk(rel, canon, ids, mask=15, per_cluster=False):
    parts = {k: [] for k, _ in KEYS}
    for k in ids:
        v = oracle.cluster_relations(canon, int(k)) if per_cluster else oracle.cluster_view(rel, canon, int(k))
        for name, okey in KEYS:
            if mask & REL[name]:
                parts[name].append(np.asarray(v[okey]).astype(np.int32))
    return {name: (np.concatenate(p) if p else np.zeros(0, np.int32)) for name, p in parts.items()
            if mask & REL[name]}


def assert_bulk_equal(got, want):
    for name in want:
        g, w = got[name], want[name]
        assert g.shape == w.shape, (name, g.shape, w.shape)
        if not np.array_equal(g, w):
            bad = np.nonzero(g != w)[0]
            raise AssertionError(f"{name}: {bad.size} mismatches, first at {bad[:5]}: got {g[bad[:5]]} want {w[bad[:5]]}")
