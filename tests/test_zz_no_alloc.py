"""The allocation-free build (gale_build_clusters_noalloc) through the C ABI.

Callers that cannot allocate device memory when they need relations (a
serving thread that must not synchronise the GPU, an application whose own
pool owns all of HBM) own the output arrays and pass them in, with their
capacities; the library's scratch for this call lives in a fixed device
array that keeps the previous call's contents.  So every case below runs
several calls in a row on one context: growing, shrinking and repeated
lists, a partial relation mask with the other arrays absent, and a
multi-bin Delaunay list.  The outputs must equal those of
gale_build_clusters and of the CPU oracle bit for bit (integer relations:
tolerance zero).  This file is collected last."""
import numpy as np
import pytest

import gen
import oracle
import paper_2507_15230_gb300 as gale
from parity_util import assert_bulk_equal, expected_bulk

pytestmark = pytest.mark.gpu


def _out_like(want, torch):
    return {n: torch.full((max(int(a.size), 1),), -7, dtype=torch.int32, device="cuda") for n, a in want.items()}


def _got(out, want):
    return {n: out[n][:a.size].cpu().numpy() for n, a in want.items()}


def test_noalloc_matches_batched_build_on_calls_in_a_row():
    import torch
    m = gen.small_grid(with_field=False)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    rng = np.random.default_rng(7)
    lists = [rng.permutation(m.nclusters)[:77].astype(np.int32),
             np.arange(m.nclusters, dtype=np.int32)[::-1].copy(),
             rng.permutation(m.nclusters)[:9].astype(np.int32)]  # shorter, after the full list
    with gale.Context.load(m, device=0) as ctx:
        for ids in lists:
            ctx.build(ids, gale.ALL, gale.MODE_BATCHED)
            ctx.synchronize()
            want = ctx.export(gale.ALL)
            out = _out_like(want, torch)
            ctx.build_noalloc(ids, gale.ALL, out)
            got = _got(out, want)
            for n, a in want.items():
                assert np.array_equal(got[n], a), n
            assert_bulk_equal(got, expected_bulk(rel, canon, ids))


def test_noalloc_partial_mask_with_absent_arrays():
    import torch
    m = gen.small_grid(with_field=False)
    mask = gale.VT | gale.TT
    ids = np.arange(0, m.nclusters, 3, dtype=np.int32)
    with gale.Context.load(m, device=0) as ctx:
        ctx.build_noalloc(np.arange(m.nclusters, dtype=np.int32), gale.ALL,
                          _out_like(ctx_full_export(ctx, m), torch))  # scratch now holds a full list
        ctx.build(ids, mask, gale.MODE_BATCHED)
        ctx.synchronize()
        want = ctx.export(mask)
        out = {n: None for n in gale.ARRAYS}
        out.update(_out_like(want, torch))
        ctx.build_noalloc(ids, mask, out)
        got = _got(out, want)
        for n, a in want.items():
            assert np.array_equal(got[n], a), n


def ctx_full_export(ctx, m):
    ctx.build(None, gale.ALL, gale.MODE_BATCHED)
    ctx.synchronize()
    return ctx.export(gale.ALL)


def test_noalloc_repeated_ids_build_each_slot():
    import torch
    m = gen.small_grid(with_field=False)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    ids = np.array([5, 17, 5, 5, 90, 17], np.int32)
    with gale.Context.load(m, device=0) as ctx:
        want = expected_bulk(rel, canon, ids)
        out = _out_like(want, torch)
        ctx.build_noalloc(ids, gale.ALL, out)
        assert_bulk_equal(_got(out, want), want)
        # each copy equals the single-id build
        for k in (5, 17, 90):
            one = expected_bulk(rel, canon, [k])
            o1 = _out_like(one, torch)
            ctx.build_noalloc(np.array([k], np.int32), gale.ALL, o1)
            assert_bulk_equal(_got(o1, one), one)


def test_noalloc_multi_bin_delaunay_list_against_oracle():
    import torch
    m = gen.delaunay_mesh(20000, seed=5, with_field=False)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    with gale.Context.load(m, device=0) as ctx:
        bins = ctx.bins()
        members = ctx.bin_members()
        starts = np.concatenate([[0], np.cumsum([b["clusters"] for b in bins])])
        K = m.nclusters  # members above K are parts of cut clusters, not cluster ids
        ok = [x[x < K] for x in (members[starts[i]:starts[i + 1]] for i, b in enumerate(bins) if not b["spill"])]
        ok = [x for x in ok if x.size]
        assert len(ok) >= 2, bins  # the list spans several shared-memory bins
        rng = np.random.default_rng(3)
        ids = rng.permutation(np.concatenate(ok)).astype(np.int32)[:600]
        for call in range(2):
            sub = ids if call == 0 else ids[::-2].copy()
            want = expected_bulk(rel, canon, sub)
            out = _out_like(want, torch)
            ctx.build_noalloc(sub, gale.ALL, out)
            assert_bulk_equal(_got(out, want), want)
        spill = [x[x < K] for x in (members[starts[i]:starts[i + 1]] for i, b in enumerate(bins) if b["spill"])]
        spill = [x for x in spill if x.size]
        if spill:
            dummy = {n: torch.zeros(1 << 20, dtype=torch.int32, device="cuda") for n in gale.ARRAYS}
            with pytest.raises(gale.GaleError) as ei:
                ctx.build_noalloc(np.array([spill[0][0]], np.int32), gale.ALL, dummy)
            assert ei.value.status == 1


def test_noalloc_rejects_bad_lists_and_short_arrays():
    import torch
    m = gen.small_grid(with_field=False)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    with gale.Context.load(m, device=0) as ctx:
        dummy = {n: torch.zeros(1, dtype=torch.int32, device="cuda") for n in gale.ARRAYS}
        with pytest.raises(gale.GaleError) as ei:
            ctx.build_noalloc(np.zeros(4097, np.int32), gale.ALL, dummy)
        assert ei.value.status == 1
        with pytest.raises(gale.GaleError):
            ctx.build_noalloc(np.array([m.nclusters], np.int32), gale.ALL, dummy)
        # one element short in one array: rejected before any launch
        ids = np.arange(10, dtype=np.int32)
        want = expected_bulk(rel, canon, ids)
        for name in ("vt_val", "et_off", "tt_val"):
            out = _out_like(want, torch)
            out[name] = torch.full((int(want[name].size) - 1,), -7, dtype=torch.int32, device="cuda")
            with pytest.raises(gale.GaleError) as ei:
                ctx.build_noalloc(ids, gale.ALL, out)
            assert ei.value.status == 1
            assert bool((out[name] == -7).all())  # nothing was written
        out = _out_like(want, torch)
        ctx.build_noalloc(ids, gale.ALL, out)
        assert_bulk_equal(_got(out, want), want)
