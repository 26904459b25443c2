"""Parity at the full sizes of the two build workloads, in the launch
configuration the benchmark times (batched, graph replay, autotuned bins):

* the 256^3 Freudenthal grid (100.7M tets, 65,536 kd leaves of <= 512
  vertices), and
* the Delaunay tetrahedralization of 2M Gaussian-mixture points (~13.5M tets,
  uneven kd leaves of 32..2,048 vertices).

The oracle cannot build whole meshes of this size in seconds, so sampled
clusters (first, last, largest, smallest, one from every size bin, random)
are compared bit-exactly with its per-cluster relations, and the whole
output is checked against properties that hold at any size: the closed-form
totals of the Freudenthal subdivision, the Euler characteristic of a
triangulated ball, every tet in exactly four VT rows, and TT symmetry."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2507_15230_gb300 as gale

pytestmark = pytest.mark.gpu


def device_arrays(ctx):
    ptrs, lens = ctx.bulk_arrays()
    return {n: gale.device_tensor(ptrs[n], lens[n]) if lens[n] else torch.empty(0, dtype=torch.int32, device="cuda")
            for n in lens}


def global_rows(off, counts):
    """Per-cluster offset segments (count+1 entries each) -> row lengths of
    the concatenated rows."""
    seg_end = torch.cumsum(torch.as_tensor(counts + 1, device=off.device), 0)
    keep = torch.ones(off.numel(), dtype=torch.bool, device=off.device)
    keep[seg_end - 1] = False
    lens = off[1:].long() - off[:-1].long()
    return lens[keep[:-1]]


def check_tt_symmetric(d, I_T):
    nt = int(I_T[-1])
    lens = global_rows(d["tt_off"], np.diff(I_T))
    assert lens.numel() == nt and int(lens.min()) >= 0 and int(lens.max()) <= 4
    row = torch.repeat_interleave(torch.arange(nt, device=lens.device), lens)
    val = d["tt_val"].long()
    assert row.numel() == val.numel()
    assert bool((val != row).all())
    fwd = torch.sort(row * nt + val).values
    bwd = torch.sort(val * nt + row).values
    assert torch.equal(fwd, bwd)
    return int(val.numel())


def _chunks(n, step=1 << 26):
    for a in range(0, n, step):
        yield a, min(n, a + step)


def _strictly_ascending_rows(owner, val):
    """Within every row (equal owner), values strictly ascending."""
    if val.numel() < 2:
        return True
    same = owner[1:] == owner[:-1]
    return bool((val[1:][same] > val[:-1][same]).all())


def check_exact(ctx, d, m):
    """Whole-output exactness of VT, VV, ET and TT, every row: each listed
    entry is valid (its tet contains the row's vertex or edge; its face
    neighbour shares three vertices), entries are distinct (rows strictly
    ascending), and the totals are the closed forms (every tet in four VT
    rows and six ET rows; VV pairs with the larger vertex second are exactly
    the ET edges; TT symmetric).  Valid and distinct entries in the right
    number leave no room for a wrong one."""
    I_V, I_T, sizes = ctx.intervals()
    nv, nt = int(I_V[-1]), int(I_T[-1])
    dev = d["vt_val"].device
    rows = torch.from_numpy(np.ascontiguousarray(ctx.rows())).to(dev).view(nt, 4)
    nvo = np.diff(I_V)
    verts = torch.arange(nv, device=dev)

    def contains(t, v):
        return bool((rows[t.long()] == v.view(-1, 1).int()).any(1).all())

    # VT: every entry a tet holding the row's vertex, rows strictly ascending
    vt_owner = torch.repeat_interleave(verts, global_rows(d["vt_off"], nvo))
    vt = d["vt_val"]
    assert vt_owner.numel() == vt.numel() == 4 * nt
    assert bool((torch.bincount(vt.long(), minlength=nt) == 4).all())  # every tet in four rows
    for a, b in _chunks(vt.numel()):
        assert contains(vt[a:b], vt_owner[a:b])
    assert _strictly_ascending_rows(vt_owner, vt)
    del vt_owner
    # ET: the edge list (lower vertex u from et_uoff, upper w), then every ET
    # entry a tet holding both endpoints
    e_u = torch.repeat_interleave(verts, global_rows(d["et_uoff"], nvo))
    e_w = d["et_w"].long()
    E = e_w.numel()
    assert e_u.numel() == E and bool((e_w > e_u).all())
    ekey = e_u * nv + e_w
    assert bool((ekey[1:] > ekey[:-1]).all())  # edges distinct, in (u, w) order
    et_len = global_rows(d["et_off"], sizes[:, 2].astype(np.int64))
    assert et_len.numel() == E and int(et_len.min()) >= 1  # every listed edge lies in some tet
    et_owner = torch.repeat_interleave(torch.arange(E, device=dev), et_len)
    et = d["et_val"]
    assert et_owner.numel() == et.numel() == 6 * nt
    for a, b in _chunks(et.numel()):
        o = et_owner[a:b]
        assert contains(et[a:b], e_u[o]) and contains(et[a:b], e_w[o])
    assert _strictly_ascending_rows(et_owner, et)
    del et_owner
    # VV: symmetric, no self loops, rows strictly ascending, and the pairs
    # (v, u) with u > v are exactly the ET edges
    vv_owner = torch.repeat_interleave(verts, global_rows(d["vv_off"], nvo))
    vv = d["vv_val"].long()
    assert vv_owner.numel() == vv.numel() == 2 * E
    assert bool((vv != vv_owner).all()) and _strictly_ascending_rows(vv_owner, vv)
    up = vv > vv_owner
    assert torch.equal(torch.sort(vv_owner[up] * nv + vv[up]).values, ekey)
    assert torch.equal(torch.sort(vv_owner * nv + vv).values, torch.sort(vv * nv + vv_owner).values)
    del vv_owner, vv, up
    # TT: every entry shares a face (three vertices) with its row's tet
    tt_owner = torch.repeat_interleave(torch.arange(nt, device=dev), global_rows(d["tt_off"], np.diff(I_T)))
    tt = d["tt_val"]
    for a, b in _chunks(tt.numel()):
        r0, r1 = rows[tt_owner[a:b]], rows[tt[a:b].long()]
        common = (r0.unsqueeze(2) == r1.unsqueeze(1)).any(2).sum(1)
        assert bool((common == 3).all())
    assert _strictly_ascending_rows(tt_owner, tt)
    return E


def check_vt_counts(d, nt):
    cnt = torch.bincount(d["vt_val"].long(), minlength=nt)
    assert cnt.numel() == nt and bool((cnt == 4).all())


def compare_sampled(ctx, canon, ks):
    for k in ks:
        k = int(k)
        got = gale.view_to_numpy(ctx.bulk_view(k))
        want = oracle.cluster_relations(canon, k)
        for g, w in [("vt_off", "vt_off"), ("vt_val", "vt_val"), ("vv_off", "vv_off"), ("vv_val", "vv_val"),
                     ("et_uoff", "eu_off"), ("et_w", "e_w"), ("et_off", "et_off"), ("et_val", "et_val"),
                     ("tt_off", "tt_off"), ("tt_val", "tt_val")]:
            assert np.array_equal(got[g].astype(np.int64), want[w].astype(np.int64)), (k, g)


def sample_clusters(ctx, canon, rng, extra):
    I_V = canon["I_V"]
    size = np.diff(I_V)
    K = size.size
    ks = {0, K - 1, int(size.argmax()), int(size.argmin())}
    # one cluster of every size bin (members above K are parts of cut
    # clusters, whose own bins list the clusters)
    order = ctx.bin_members()
    start = 0
    for b in ctx.bins():
        mem = order[start:start + b["clusters"]]
        mem = mem[mem < K]
        if mem.size:
            ks.add(int(mem[0]))
        start += b["clusters"]
    ks.update(int(k) for k in rng.choice(K, extra, replace=False))
    return sorted(ks)


def test_grid256_full_size():
    n = 256
    m = gen.scale_grid(n)
    with gale.Context.load(m, device=0) as ctx:
        ctx.autotune(gale.ALL, reps=1)
        for _ in range(2):  # the second build replays the captured graph
            ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        d = device_arrays(ctx)
        T, V = 6 * n ** 3, (n + 1) ** 3
        E = 7 * n ** 3 + 9 * n ** 2 + 3 * n
        assert d["vt_val"].numel() == 4 * T
        assert d["vv_val"].numel() == 2 * E
        assert d["et_w"].numel() == E
        assert d["et_val"].numel() == 6 * T
        assert d["tt_val"].numel() == 4 * T - 12 * n ** 2
        I_V, I_T, _ = ctx.intervals()
        check_vt_counts(d, T)
        check_tt_symmetric(d, I_T)
        assert check_exact(ctx, d, m) == E
        del d
        torch.cuda.empty_cache()
        canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
        assert np.array_equal(canon["I_V"], I_V) and np.array_equal(canon["I_T"], I_T)
        compare_sampled(ctx, canon, sample_clusters(ctx, canon, np.random.default_rng(7), 6))


def test_delaunay_2m_full_size():
    """Besides the whole-output properties and sampled clusters, the largest
    clusters - cut into parts that batched builds run one CTA each - are
    checked in the batched, per-cluster and served forms."""
    import threading
    m = gen.delaunay_mesh(2_000_000, seed=5, with_field=False)
    with gale.Context.load(m, device=0, cache_budget_bytes=1 << 30) as ctx:
        bins0 = ctx.bins()
        assert ctx.info().nparts > 0, bins0
        assert any(b["parts"] > 0 for b in bins0), bins0
        cut = [i for i, b in enumerate(bins0) if b["parts"] == -1]
        assert cut, bins0
        members = ctx.bin_members()
        starts = np.concatenate([[0], np.cumsum([b["clusters"] for b in bins0])])
        pi_ids = np.concatenate([members[starts[i]:starts[i + 1]] for i in cut])
        ctx.autotune(gale.ALL, reps=1)
        assert [b["parts"] for b in ctx.bins()] == [b["parts"] for b in bins0]
        for _ in range(2):
            ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        d = device_arrays(ctx)
        T, V = m.nt, m.nv
        E = d["et_w"].numel()
        assert d["vt_val"].numel() == 4 * T
        assert d["vv_val"].numel() == 2 * E
        assert d["et_val"].numel() == 6 * T
        I_V, I_T, _ = ctx.intervals()
        check_vt_counts(d, T)
        sum_tt = check_tt_symmetric(d, I_T)
        # faces: interior ones are counted twice by TT, boundary ones not at
        # all, so F = 4T - sum|TT|/2; a triangulated ball has V - E + F - T = 1
        F = 4 * T - sum_tt // 2
        assert V - E + F - T == 1
        assert check_exact(ctx, d, m) == E
        del d
        torch.cuda.empty_cache()
        canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
        assert np.array_equal(canon["I_V"], I_V) and np.array_equal(canon["I_T"], I_T)
        rng = np.random.default_rng(11)
        compare_sampled(ctx, canon, sample_clusters(ctx, canon, rng, 10))
        picks = sorted(int(k) for k in rng.choice(pi_ids, 12, replace=False))
        compare_sampled(ctx, canon, picks)
        # the same clusters, one launch each, then served by gale_request
        sub = np.array(picks, np.int32)
        ctx.build(sub, gale.ALL, gale.MODE_PER_CLUSTER)
        ctx.synchronize()
        want = {k: oracle.cluster_relations(canon, k) for k in picks}
        keys = [("vt_off", "vt_off"), ("vt_val", "vt_val"), ("vv_off", "vv_off"), ("vv_val", "vv_val"),
                ("et_uoff", "eu_off"), ("et_w", "e_w"), ("et_off", "et_off"), ("et_val", "et_val"),
                ("tt_off", "tt_off"), ("tt_val", "tt_val")]
        for i, k in enumerate(picks):
            got = gale.view_to_numpy(ctx.bulk_view(i))
            for g, w in keys:
                assert np.array_equal(got[g].astype(np.int64), want[k][w].astype(np.int64)), (k, g)
        errors = []

        def consumer(ks):
            for k in ks:
                v = ctx.request(k, gale.ALL, timeout_ns=60_000_000_000)
                got = gale.view_to_numpy(v)
                ctx.release(v)
                if not all(np.array_equal(got[g].astype(np.int64), want[k][w].astype(np.int64)) for g, w in keys):
                    errors.append(k)

        th = [threading.Thread(target=consumer, args=(picks[j::3],)) for j in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors, errors


def test_exactness_checks_catch_planted_mistakes():
    """The whole-output checks above pass on a correct build and fail on
    copies of it with one planted mistake each: a VT entry moved to another
    tet, two ET entries swapped across rows, a VV entry replaced, a TT
    neighbour replaced."""
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=0) as ctx:
        ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        d = {n: t.clone() for n, t in device_arrays(ctx).items()}
        check_exact(ctx, d, m)

        def planted(name, fn):
            bad = {n: t.clone() for n, t in d.items()}
            fn(bad[name])
            with pytest.raises(AssertionError):
                check_exact(ctx, bad, m)

        def vt_move(a):
            a[10] = (a[10] + 1) % m.tv.shape[0]

        def et_swap(a):
            i, j = 3, a.numel() // 2
            a[i], a[j] = a[j].clone(), a[i].clone()

        def vv_replace(a):
            a[7] = a[8]

        def tt_replace(a):
            a[5] = (a[5] + 7) % m.tv.shape[0]

        planted("vt_val", vt_move)
        planted("et_val", et_swap)
        planted("vv_val", vv_replace)
        planted("tt_val", tt_replace)
