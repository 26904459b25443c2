"""C ABI checks that need no GPU: the library loads and exports every symbol
include/gale.h declares, and the host-side initialisation (input checks,
canonical numbering, I_V / I_T, T_ex and halo working sets; Section 4.3) of
a host-only context matches the oracle exactly."""
import os
import re

import numpy as np
import pytest

import gen
import oracle
import paper_2507_15230_gb300 as gale

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gale.h")).read()
    return sorted(set(re.findall(r"\b(gale_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = gale.load_library()
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(gale.EXPORTS)


def host_ctx(m, mask=gale.ALL):
    return gale.Context.load(m, precondition_mask=mask, device=-1)


def compare_with_oracle(m, ctx):
    canon = oracle.canonicalize(m.nv if hasattr(m, "nv") else m.seg.shape[0], m.tv, m.seg, m.nclusters)
    vp, tp = ctx.permutations()
    assert np.array_equal(vp, canon["vperm"])
    assert np.array_equal(tp, canon["tperm"])
    I_V, I_T, _ = ctx.intervals()
    assert np.array_equal(I_V, canon["I_V"])
    assert np.array_equal(I_T, canon["I_T"])
    assert np.array_equal(ctx.rows(), canon["rows"])
    return canon


def test_host_init_small_matches_oracle(small_mesh):
    m = small_mesh
    with host_ctx(m) as ctx:
        canon = compare_with_oracle(m, ctx)
        for k in range(m.nclusters):
            ext, halo = ctx.working_set(k)
            oext, ohalo = oracle.working_set(canon, k)
            assert np.array_equal(ext, oext), k
            assert np.array_equal(halo, ohalo), k
        info = ctx.info()
        assert info.nv == m.nv and info.nt == m.nt and info.nclusters == m.nclusters


@pytest.mark.parametrize("n,K", [(2, 1), (3, 5), (3, 64), (4, 7)])
def test_host_init_random_partitions(n, K):
    xyz, tv = gen.freudenthal_grid(n, permute=True, seed=11 * n + K)
    nv = xyz.shape[0]
    rng = np.random.default_rng(n * 100 + K)
    seg = rng.integers(0, K, nv).astype(np.int32)
    seg[:K] = np.arange(K)
    m = gen.Mesh(xyz, tv, seg, K)
    with host_ctx(m) as ctx:
        canon = compare_with_oracle(m, ctx)
        for k in range(K):
            ext, halo = ctx.working_set(k)
            oext, ohalo = oracle.working_set(canon, k)
            assert np.array_equal(ext, oext) and np.array_equal(halo, ohalo), k


def test_host_init_rejects_bad_input():
    tv = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], np.int32)
    seg = np.array([0, 0, 1, 1, 1], np.int32)
    ok = gen.Mesh(None, tv, seg, 2)
    host_ctx(ok).close()
    bad = [
        gen.Mesh(None, np.array([[0, 1, 2, 5]], np.int32), seg, 2),
        gen.Mesh(None, np.array([[0, 1, 1, 3]], np.int32), seg, 2),
        gen.Mesh(None, np.array([[0, 1, 2, 3], [3, 2, 1, 0]], np.int32), seg, 2),
        gen.Mesh(None, tv, np.array([0, 0, 2, 1, 1], np.int32), 2),
    ]
    for m in bad:
        assert oracle.validate(5, m.tv, m.seg, m.nclusters) == oracle.EINVAL
        with pytest.raises(gale.GaleError) as ei:
            host_ctx(m)
        assert ei.value.status == 1
    with pytest.raises(gale.GaleError):
        host_ctx(ok, mask=0)


def test_host_init_delaunay_matches_oracle():
    m = gen.delaunay_mesh(6000, seed=3, with_field=False)
    with host_ctx(m) as ctx:
        canon = compare_with_oracle(m, ctx)
        for k in range(0, m.nclusters, max(1, m.nclusters // 12)):
            ext, halo = ctx.working_set(k)
            oext, ohalo = oracle.working_set(canon, k)
            assert np.array_equal(ext, oext) and np.array_equal(halo, ohalo), k


def test_copy_to_host_refuses_host_only_and_null(small_mesh):
    """gale_copy_to_host needs a device context and non-NULL pointers; a
    zero-byte copy of NULL is still refused on a host-only context."""
    lib = gale.load_library()
    with host_ctx(small_mesh) as ctx:
        buf = np.zeros(4, np.int32)
        assert lib.gale_copy_to_host(ctx._h, buf.ctypes.data, None, 16) == 1  # EINVAL
        assert lib.gale_copy_to_host(ctx._h, None, None, 0) == 1  # EINVAL
        assert lib.gale_copy_to_host(None, buf.ctypes.data, 1, 16) == 1  # EINVAL
        with pytest.raises(gale.GaleError):
            ctx.copy_to_host(1 << 20, 4, out=buf)


def test_host_init_local_id_limits():
    """A cluster's working set is packed with 16-bit local ids: at most
    65535 local vertices and 65534 tets.  A single cluster just under the
    tet limit loads; one over it, or one with more local vertices than
    the limit, is rejected with EINVAL naming the cluster."""
    def one_cluster(tv, nv):
        return gen.Mesh(None, tv.astype(np.int32), np.zeros(nv, np.int32), 1)

    _, tv = gen.freudenthal_grid(22, permute=True, seed=3)  # 63,888 tets
    host_ctx(one_cluster(tv, 23 ** 3)).close()
    _, tv = gen.freudenthal_grid(23, permute=True, seed=3)  # 73,002 tets
    with pytest.raises(gale.GaleError) as ei:
        host_ctx(one_cluster(tv, 24 ** 3))
    assert ei.value.status == 1 and "cluster 0" in str(ei.value)
    nt = 16_400  # disjoint tets: 65,600 vertices
    tv = np.arange(4 * nt, dtype=np.int32).reshape(nt, 4)
    with pytest.raises(gale.GaleError) as ei:
        host_ctx(one_cluster(tv, 4 * nt))
    assert ei.value.status == 1 and "65535" in str(ei.value)
