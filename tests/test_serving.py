"""Serving (gale_request / gale_release): continuous batching through the
device-resident loop (or the launch-per-batch mode), the HBM-budgeted LRU
cache, admission against the budget, and the critical-point consumer.

Every served result must equal the CPU oracle's relations of that cluster,
bit for bit, whatever else is in flight; the same cluster built alone by the
bulk path is checked as well ("the same alone and in the mix")."""
import os
import threading

import numpy as np
import pytest

import gen
import oracle
import paper_2507_15230_gb300 as gale
from parity_util import expected_bulk

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bulk_reference(ctx, mask=gale.ALL):
    """Per-cluster relations from the bulk path, each cluster built alone."""
    ref = {}
    for k in range(ctx.K):
        ctx.build(np.array([k], np.int32), mask, gale.MODE_BATCHED)
        ctx.synchronize()
        ref[k] = gale.view_to_numpy(ctx.bulk_view(0))
    return ref


def same(a, b):
    return a.keys() == b.keys() and all(np.array_equal(a[n], b[n]) for n in a)


def oracle_reference(m, mask=gale.ALL):
    """Per-cluster relations of the CPU oracle (global definitions, sliced
    per cluster), in the layout of a served view."""
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    return {k: expected_bulk(rel, canon, [k], mask) for k in range(m.nclusters)}


def run_mix(budget, nthreads=8, rounds=40, masks=(gale.ALL, gale.VT | gale.VV | gale.TT, gale.ET),
            mode=gale.SERVE_LOOP):
    m = gen.small_grid(with_field=False)
    orefs = {mk: oracle_reference(m, mk) for mk in masks}
    with gale.Context.load(m, device=0, cache_budget_bytes=budget) as ctx:
        ctx.serve_configure(mode)
        refs = {mk: bulk_reference(ctx, mk) for mk in masks}
        for mk in masks:  # alone = the oracle
            for k in range(ctx.K):
                assert same(refs[mk][k], orefs[mk][k]), (mk, k)
        errors = []

        def consumer(seed):
            rng = np.random.default_rng(seed)
            for _ in range(rounds):
                k = int(rng.integers(ctx.K))
                mk = masks[int(rng.integers(len(masks)))]
                v = ctx.request(k, mk, timeout_ns=20_000_000_000)
                got = gale.view_to_numpy(v)
                want = {n: a for n, a in refs[mk][k].items()}
                # a cached superset entry may serve a narrower mask
                got = {n: got[n] for n in want}
                if not same(got, want) or not same(got, orefs[mk][k]):
                    errors.append((k, mk))
                ctx.release(v)

        th = [threading.Thread(target=consumer, args=(i,)) for i in range(nthreads)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        stats = ctx.serve_stats()
        return errors, stats


@pytest.mark.parametrize("mode", [gale.SERVE_LOOP, gale.SERVE_BATCH, gale.SERVE_SINGLE])
def test_results_same_alone_and_in_mix(mode):
    errors, stats = run_mix(64 << 20, mode=mode)
    assert not errors
    assert stats.requests == 8 * 40 and stats.builds > 0 and stats.hits > 0


def test_lru_evicts_under_tiny_budget():
    errors, stats = run_mix(256 << 10, nthreads=4, rounds=30)
    assert not errors
    assert stats.evictions > 0
    assert stats.cache_bytes_used <= 256 << 10


def entry_bytes(ctx, k):
    """Cache footprint of one cluster's four relations (16-byte aligned
    arrays, 256-byte aligned entry)."""
    I_V, I_T, sizes = ctx.intervals()
    nvo, nown = int(I_V[k + 1] - I_V[k]), int(I_T[k + 1] - I_T[k])
    vt, vv, ne, et, tt = (int(x) for x in sizes[k])
    lens = [nvo + 1, vt, nvo + 1, vv, nvo + 1, ne, ne + 1, et, nown + 1, tt]
    b = sum((4 * n + 15) // 16 * 16 for n in lens)
    return (b + 255) // 256 * 256


def test_admission_waits_for_release():
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=0) as probe:
        sz = [entry_bytes(probe, k) for k in range(3)]
    budget = sz[0] + sz[1] + min(sz[2], min(sz[0], sz[1])) // 2  # two fit, not three
    with gale.Context.load(m, device=0, cache_budget_bytes=budget) as ctx:
        a = ctx.request(0, gale.ALL, timeout_ns=10_000_000_000)
        b = ctx.request(1, gale.ALL, timeout_ns=10_000_000_000)
        got = {}

        def late():
            got["v"] = ctx.request(2, gale.ALL, timeout_ns=20_000_000_000)

        t = threading.Thread(target=late)
        t.start()
        t.join(timeout=1.0)
        blocked = t.is_alive()
        ctx.release(a)
        ctx.release(b)
        t.join(timeout=20)
        assert blocked and "v" in got
        ctx.release(got["v"])
        assert ctx.serve_stats().evictions >= 1


def test_serve_configure_after_start_is_busy():
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=0, cache_budget_bytes=8 << 20) as ctx:
        ctx.release(ctx.request(3, gale.VT))
        with pytest.raises(gale.GaleError) as ei:
            ctx.serve_configure(gale.SERVE_BATCH)
        assert ei.value.status == 3


def test_oversized_request_is_rejected():
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=0, cache_budget_bytes=4096) as ctx:
        with pytest.raises(gale.GaleError) as ei:
            ctx.request(0, gale.ALL, timeout_ns=5_000_000_000)
        assert ei.value.status == 2


def test_serving_driver_matches_oracle_classification():
    import consumers
    import oracle
    m = gen.small_grid(with_field=True)
    with gale.Context.load(m, device=0, cache_budget_bytes=8 << 20) as ctx:
        vperm, _ = ctx.permutations()
        f_c, inid = consumers.canonical_inputs(m.field, vperm)
        rows = ctx.rows()
        I_V, _, _ = ctx.intervals()
        cls, lat, st = consumers.serve_run(ctx, f_c, inid, rows, I_V, nthreads=8, mask=gale.VT | gale.VV | gale.TT)
        assert st["failures"] == 0 and st["requests"] == ctx.K
        assert np.all(lat > 0)
    canon, rel = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    want = np.empty(m.nv, np.int8)
    for k in range(m.nclusters):
        v = oracle.cluster_view(rel, canon, k)
        want[canon["I_V"][k]:canon["I_V"][k + 1]] = consumers.classify_cluster(
            f_c, inid, canon["rows"], canon["I_V"][k], v["vt_off"], v["vt_val"], v["vv_off"], v["vv_val"])
    assert np.array_equal(cls, want)


def test_mixed_meshes_loops_side_by_side():
    """Four loaded meshes (two grids, two Delaunay meshes), each with its own
    device loop capped at 8 CTAs so all stay resident, serve requests for
    random (mesh, cluster, mask) from 12 threads under small budgets; every
    result equals that mesh's bulk build of the cluster, bit for bit."""
    meshes = [gen.freudenthal_mesh(6, 64, seed=7, jitter=0.3, with_field=False),
              gen.freudenthal_mesh(9, 64, seed=8, jitter=0.3, with_field=False),
              gen.delaunay_mesh(3000, seed=18, kd_cap=512, with_field=False),
              gen.delaunay_mesh(6000, seed=19, kd_cap=512, with_field=False)]
    orefs = [oracle_reference(m) for m in meshes]
    ctxs = [gale.Context.load(m, device=0, cache_budget_bytes=1 << 20) for m in meshes]
    try:
        refs = [bulk_reference(c) for c in ctxs]
        for r, o in zip(refs, orefs):
            assert all(same(r[k], o[k]) for k in o)
        for c in ctxs:
            c.serve_configure(gale.SERVE_LOOP, loop_ctas=8)
        names = {gale.VT: ("vt_off", "vt_val"), gale.VV: ("vv_off", "vv_val"),
                 gale.ET: ("et_uoff", "et_w", "et_off", "et_val"), gale.TT: ("tt_off", "tt_val")}
        errors = []

        def consumer(seed):
            rng = np.random.default_rng(seed)
            for _ in range(40):
                i = int(rng.integers(len(ctxs)))
                k = int(rng.integers(ctxs[i].K))
                mk = int(rng.integers(1, 16))
                v = ctxs[i].request(k, mk, timeout_ns=20_000_000_000)
                got = gale.view_to_numpy(v)
                for bit, arrs in names.items():
                    if mk & bit:
                        for n in arrs:
                            if not np.array_equal(got[n], refs[i][k][n]) or not np.array_equal(got[n], orefs[i][k][n]):
                                errors.append((i, k, mk, n))
                ctxs[i].release(v)

        th = [threading.Thread(target=consumer, args=(s,)) for s in range(12)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors, errors[:5]
        st = [c.serve_stats() for c in ctxs]
        assert sum(s.requests for s in st) == 12 * 40
        assert all(s.cache_bytes_used <= 1 << 20 for s in st)
        # the native open-loop driver over the same meshes: Poisson arrivals
        import consumers
        rng = np.random.default_rng(4)
        n = 400
        mi = rng.integers(len(ctxs), size=n)
        ks = np.array([rng.integers(ctxs[i].K) for i in mi])
        masks = rng.integers(1, 16, size=n)
        lat, wall, fails, first = consumers.open_loop(ctxs, mi, ks, masks, rate=20000.0, seed=9, workers=16)
        assert fails == 0 and first == -1
        assert lat.shape == (n,) and (lat >= 0).all() and wall > 0
        assert sum(c.serve_stats().requests for c in ctxs) == 12 * 40 + n
    finally:
        for c in ctxs:
            c.close()


def test_loop_mode_with_clusters_too_large_for_it():
    """A Delaunay mesh whose largest clusters run in global scratch: the loop
    serves the size bins that fit it and the leader builds the rest by
    batched launches beside it; every result equals the bulk build."""
    m = gen.delaunay_mesh(60000, seed=11, with_field=False)
    oref = oracle_reference(m)
    with gale.Context.load(m, device=0, cache_budget_bytes=64 << 20) as ctx:
        assert any(b["spill"] for b in ctx.bins())
        ref = bulk_reference(ctx)
        assert all(same(ref[k], oref[k]) for k in oref)
        ctx.serve_configure(gale.SERVE_LOOP, loop_ctas=16)
        I_V, _, _ = ctx.intervals()
        size = np.diff(I_V)
        big = [int(k) for k in np.argsort(size)[-6:]]
        errors = []

        def consumer(seed):
            rng = np.random.default_rng(seed)
            picks = big + [int(k) for k in rng.integers(ctx.K, size=20)]
            for k in picks:
                v = ctx.request(k, gale.ALL, timeout_ns=60_000_000_000)
                got = gale.view_to_numpy(v)
                if not same(got, ref[k]) or not same(got, oref[k]):
                    errors.append(k)
                ctx.release(v)

        th = [threading.Thread(target=consumer, args=(s,)) for s in range(6)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors
        assert ctx.serve_stats().requests == 6 * 26


@pytest.mark.parametrize("mode", [gale.SERVE_LOOP, gale.SERVE_BATCH])
def test_prefetch_serves_following_clusters(mode):
    """With prefetch depth 3, a request for cluster k also queues k+1..k+3;
    consumers walking in cluster order then find their next clusters already
    built or in flight.  Every result still equals the bulk build."""
    m = gen.small_grid(with_field=False)
    oref = oracle_reference(m)
    with gale.Context.load(m, device=0, cache_budget_bytes=64 << 20) as ctx:
        ref = bulk_reference(ctx)
        assert all(same(ref[k], oref[k]) for k in oref)
        ctx.serve_configure(mode, prefetch=3)
        errors = []

        def walker(start):
            for k in range(start, min(start + 24, ctx.K)):
                v = ctx.request(k, gale.ALL, timeout_ns=20_000_000_000)
                if not same(gale.view_to_numpy(v), ref[k]):
                    errors.append(k)
                ctx.release(v)

        th = [threading.Thread(target=walker, args=(s,)) for s in (0, 32, 64, 96)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors
        st = ctx.serve_stats()
        assert st.requests == 4 * 24
        assert st.prefetches > 0 and st.prefetch_hits > 0
        assert st.prefetch_hits + st.misses <= st.requests + st.prefetches


def test_prefetch_is_dropped_under_a_pinned_budget():
    """Prefetches never wait for the budget: with most of it pinned by held
    views they are dropped, and the held requests still complete."""
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=0, cache_budget_bytes=96 << 10) as ctx:
        ctx.serve_configure(gale.SERVE_LOOP, prefetch=8)
        held = []
        for k in (0, 40, 80):
            try:
                held.append(ctx.request(k, gale.ALL, timeout_ns=5_000_000_000))
            except gale.GaleError:
                break
        assert held
        st = ctx.serve_stats()
        assert st.prefetches > 0
        for v in held:
            ctx.release(v)
        v = ctx.request(1, gale.ALL, timeout_ns=5_000_000_000)
        ctx.release(v)


def test_lease_unpins_the_views_of_a_dead_consumer():
    """A consumer thread that exits holding views (the failure is made on the
    host: the thread simply ends) does not keep the budget pinned once the
    lease runs out; its stale views can no longer be released."""
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=0) as probe:
        sz = [entry_bytes(probe, k) for k in range(3)]
    budget = sz[0] + sz[1] + min(sz[2], min(sz[0], sz[1])) // 2  # two fit, not three
    with gale.Context.load(m, device=0, cache_budget_bytes=budget) as ctx:
        ctx.serve_set_lease(300_000_000)  # 0.3 s
        dead = {}

        def consumer():
            dead["a"] = ctx.request(0, gale.ALL, timeout_ns=10_000_000_000)
            dead["b"] = ctx.request(1, gale.ALL, timeout_ns=10_000_000_000)
            # ends without gale_release

        t = threading.Thread(target=consumer)
        t.start()
        t.join(timeout=30)
        assert "b" in dead
        v = ctx.request(2, gale.ALL, timeout_ns=20_000_000_000)  # admitted once the lease has run out
        ctx.release(v)
        st = ctx.serve_stats()
        assert st.leases_expired >= 2 and st.evictions >= 1
        for stale in (dead["a"], dead["b"]):
            with pytest.raises(gale.GaleError) as ei:
                ctx.release(stale)
            assert gale.STATUS[ei.value.status] == "ENOTFOUND"


def test_release_twice_is_rejected_without_touching_the_entry():
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=0, cache_budget_bytes=8 << 20) as ctx:
        v = ctx.request(5, gale.VT | gale.VV, timeout_ns=10_000_000_000)
        copy = gale.View.from_buffer_copy(v)
        w = ctx.request(5, gale.VT | gale.VV, timeout_ns=10_000_000_000)  # a second pin of the same entry
        ctx.release(v)
        with pytest.raises(gale.GaleError) as ei:
            ctx.release(copy)  # the same pin again
        assert gale.STATUS[ei.value.status] == "ENOTFOUND"
        ctx.release(w)  # the other pin is still valid
        with pytest.raises(gale.GaleError):
            ctx.serve_set_lease(-1)


def test_wait_breakdown_is_consistent():
    """The per-stage waiting times (Section 5.3's breakdown) are non-negative
    and bounded by the requests' total wait."""
    import consumers
    m = gen.small_grid(with_field=True)
    with gale.Context.load(m, device=0, cache_budget_bytes=64 << 20) as ctx:
        vperm, _ = ctx.permutations()
        f_c, inid = consumers.canonical_inputs(m.field, vperm)
        I_V, _, _ = ctx.intervals()
        _, lat, st = consumers.serve_run(ctx, f_c, inid, ctx.rows(), I_V, nthreads=4,
                                         mask=gale.VT | gale.VV | gale.TT)
        s = ctx.serve_stats()
        parts = (s.t_enqueue_ns, s.t_queue_ns, s.t_prepare_ns, s.t_build_ns)
        assert all(p >= 0 for p in parts) and s.t_build_ns > 0
        assert s.t_queue_ns + s.t_prepare_ns + s.t_build_ns <= s.t_wait_ns + 1_000_000
        assert 0 < s.max_wait_ns <= s.t_wait_ns
        assert 0 < s.t_kernel_ns <= s.t_build_ns + 1_000_000  # the build alone, inside the device stage
        assert abs(s.t_wait_ns * 1e-9 - float(lat.sum())) < 0.5 * float(lat.sum()) + 0.05
        assert st["copy_s"] > 0 and st["integrate_s"] > 0
        hist = list(s.depth_hist)
        assert sum(hist) > 0 and all(h >= 0 for h in hist)
        assert sum(hist[5:]) == 0  # 4 consumer threads, no prefetch: never 32 or more pending


def test_idle_loop_wait_runs_out_and_the_context_stays_usable():
    """The device loop's CTAs wait on the ring tail, a flag that nothing sets
    while no request comes; that wait is bounded by the idle limit, after
    which the loop returns by itself.  The next request relaunches it."""
    import time
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=0, cache_budget_bytes=8 << 20) as ctx:
        ctx.serve_configure(gale.SERVE_LOOP, idle_us=2000)
        ctx.release(ctx.request(0, gale.VT, timeout_ns=10_000_000_000))
        first = ctx.serve_stats().batches
        assert first >= 1
        time.sleep(0.3)  # far past the 2 ms idle limit: the loop has returned
        ctx.release(ctx.request(1, gale.VT, timeout_ns=10_000_000_000))
        st = ctx.serve_stats()
        assert st.batches == first + 1 and st.builds == 2
        ctx.synchronize()


def test_served_rows_match_the_bulk_build_at_128cubed():
    """At the 128^3 grid (12.6M tets, 8,192 clusters): 16 threads request a
    random sample of clusters under every relation mask through the device
    loop, with a budget that forces evictions; every served view equals the
    same cluster from one bulk build of all clusters, bit for bit."""
    m = gen.freudenthal_mesh(128, 512, seed=3, field_seed=4, jitter=0.3, with_field=False)
    rng = np.random.default_rng(8)
    with gale.Context.load(m, device=0, cache_budget_bytes=64 << 20) as ctx:
        ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        bulk = ctx.export(gale.ALL)
        offs = [ctx.bulk_offsets(k) for k in range(ctx.K)]
        I_V, I_T, sizes = ctx.intervals()
        sample = rng.choice(ctx.K, 400, replace=False)
        masks = list(range(1, 16))

        def want(k, mk):
            nvo, nown, ne = int(I_V[k + 1] - I_V[k]), int(I_T[k + 1] - I_T[k]), int(sizes[k, 2])
            lens = {"vt_off": nvo + 1, "vt_val": sizes[k, 0], "vv_off": nvo + 1, "vv_val": sizes[k, 1],
                    "et_uoff": nvo + 1, "et_w": ne, "et_off": ne + 1, "et_val": sizes[k, 3], "tt_off": nown + 1,
                    "tt_val": sizes[k, 4]}
            rel = {"vt_off": gale.VT, "vt_val": gale.VT, "vv_off": gale.VV, "vv_val": gale.VV, "et_uoff": gale.ET,
                   "et_w": gale.ET, "et_off": gale.ET, "et_val": gale.ET, "tt_off": gale.TT, "tt_val": gale.TT}
            return {n: bulk[n][offs[k][n]:offs[k][n] + int(lens[n])] for n in lens if mk & rel[n]}

        errors = []

        def consumer(seed):
            r = np.random.default_rng(seed)
            for k in r.permutation(sample)[:100]:
                mk = masks[int(r.integers(len(masks)))]
                v = ctx.request(int(k), mk, timeout_ns=60_000_000_000)
                got = gale.view_to_numpy(v)
                w = want(int(k), mk)
                if not same({n: got[n] for n in w}, w):
                    errors.append((int(k), mk))
                ctx.release(v)

        th = [threading.Thread(target=consumer, args=(i,)) for i in range(16)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        st = ctx.serve_stats()
        # a sample of the served clusters, fresh from the loop, against the
        # oracle's per-cluster producer
        canon = oracle.canonicalize(m.nv, m.tv, m.seg, m.nclusters)
        for k in (int(x) for x in sample[:8]):
            want_o = expected_bulk(None, canon, [k], gale.ALL, per_cluster=True)
            v = ctx.request(k, gale.ALL, timeout_ns=60_000_000_000)
            got = gale.view_to_numpy(v)
            ctx.release(v)
            assert same(got, want_o), k
    assert not errors, errors[:5]
    assert st.requests == 1600 and st.evictions > 0


def test_request_promotes_a_queued_prefetch_and_null_consumers_walk_every_cluster():
    """With a deep prefetch, requests for clusters that are still queued as
    prefetches move them to the request queue; null consumers (view taken and
    released, no work) walk every cluster, and a final sample of views equals
    the oracle."""
    import consumers
    m = gen.small_grid(with_field=True)
    oref = oracle_reference(m)
    with gale.Context.load(m, device=0, cache_budget_bytes=64 << 20) as ctx:
        ctx.serve_configure(gale.SERVE_LOOP, prefetch=8, loop_ctas=2)
        vperm, _ = ctx.permutations()
        f_c, inid = consumers.canonical_inputs(m.field, vperm)
        I_V, _, _ = ctx.intervals()
        _, lat, st = consumers.serve_run(ctx, f_c, inid, ctx.rows(), I_V, nthreads=8,
                                         mask=gale.VT | gale.VV | gale.TT, null_work=True)
        assert st["failures"] == 0 and st["requests"] == ctx.K and (lat > 0).all()
        s = ctx.serve_stats()
        assert s.prefetches > 0 and s.prefetch_hits > 0
        for k in range(0, ctx.K, 7):
            v = ctx.request(k, gale.ALL, timeout_ns=20_000_000_000)
            got = gale.view_to_numpy(v)
            ctx.release(v)
            assert same(got, oref[k]), k
