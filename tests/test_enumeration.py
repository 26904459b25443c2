"""Edge and triangle enumeration and boundary relations through the C ABI
(host work, so host-only contexts and no GPU), against the oracle: the
paper's worked example, random partitions of Freudenthal grids and a small
Delaunay mesh, both numberings, every FE / TE / TF row."""
import json
import os

import numpy as np
import pytest

import gen
import oracle
import paper_2507_15230_gb300 as gale

HERE = os.path.dirname(os.path.abspath(__file__))
ORDERS = [(gale.ENUM_SORTED, "sorted"), (gale.ENUM_FIRST_APPEARANCE, "first")]


def check_against_oracle(m, order, oname):
    canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
    want = oracle.enumerate_simplices(canon, oname)
    with gale.Context.load(m, device=-1) as ctx:
        got = ctx.enumerate(order)
        assert [tuple(e) for e in got["E"].tolist()] == want["E"]
        assert [tuple(f) for f in got["F"].tolist()] == want["F"]
        assert got["I_E"].tolist() == want["I_E"] and got["I_F"].tolist() == want["I_F"]
        nt = canon["rows"].shape[0]
        fe = ctx.boundary(gale.REL_FE, np.arange(len(want["F"])))
        assert fe.tolist() == oracle.boundary(canon, want, "FE", range(len(want["F"])))
        te = ctx.boundary(gale.REL_TE, np.arange(nt))
        assert te.tolist() == oracle.boundary(canon, want, "TE", range(nt))
        tf = ctx.boundary(gale.REL_TF, np.arange(nt))
        assert tf.tolist() == oracle.boundary(canon, want, "TF", range(nt))


def test_paper_example():
    with open(os.path.join(HERE, "golden", "mesh_input_example.json")) as f:
        g = json.load(f)
    m = gen.Mesh(np.zeros((g["nv"], 3), np.float32), np.array(g["tv"], np.int32), np.array(g["seg"], np.int32),
                 g["nclusters"])
    with gale.Context.load(m, device=-1) as ctx:
        en = ctx.enumerate(gale.ENUM_FIRST_APPEARANCE)
        assert en["I_E"].tolist() == g["expect"]["I_E"]
        assert en["F"][5].tolist() == g["expect"]["f5"]
        assert ctx.boundary(gale.REL_FE, [5]).tolist() == [g["expect"]["FE_f5"]]
        en = ctx.enumerate(gale.ENUM_SORTED)
        f5 = [tuple(x) for x in en["F"].tolist()].index(tuple(g["expect"]["f5"]))
        assert ctx.boundary(gale.REL_FE, [f5]).tolist() == [[2, 3, 9]]


@pytest.mark.parametrize("order,oname", ORDERS)
@pytest.mark.parametrize("n,K,seed", [(2, 1, 0), (3, 4, 1), (4, 11, 2), (5, 40, 3)])
def test_random_partitions(order, oname, n, K, seed):
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=seed + 60)
    seg = np.random.default_rng(seed).integers(0, K, xyz.shape[0]).astype(np.int32)
    check_against_oracle(gen.Mesh(xyz, tv, seg, K), order, oname)


@pytest.mark.parametrize("order,oname", ORDERS)
def test_delaunay(order, oname):
    check_against_oracle(gen.delaunay_mesh(2500, seed=31, kd_cap=256, with_field=False), order, oname)


def test_errors():
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=-1) as ctx:
        with pytest.raises(gale.GaleError) as ei:
            ctx.boundary(gale.REL_FE, [0])
        assert gale.STATUS[ei.value.status] == "ENOTFOUND"
        with pytest.raises(gale.GaleError):
            ctx.enumerate(7)
        en = ctx.enumerate(gale.ENUM_SORTED)
        with pytest.raises(gale.GaleError) as ei:
            ctx.boundary(gale.REL_TE, [m.nt])
        assert gale.STATUS[ei.value.status] == "EINVAL"
        with pytest.raises(gale.GaleError):
            ctx.boundary(gale.REL_FE, [len(en["F"])])
        # closed forms of the 16^3 grid
        n = 16
        assert len(en["E"]) == 7 * n ** 3 + 9 * n ** 2 + 3 * n and len(en["F"]) == 12 * n ** 3 + 6 * n ** 2
