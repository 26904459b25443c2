"""Several small clusters per CTA ("teams"), against the CPU oracle bit for
bit.

With gale_set_teams every size bin of whole clusters in shared memory runs,
in batched builds, `teams` clusters per CTA at once, one team of
team_threads threads each with barriers of its own.  The builds must equal
the oracle's relations for every team size, in full and partial builds,
every mask, the pipelined export and after the autotuner; the per-cluster
form keeps one cluster per CTA under the team-sized plan."""
import numpy as np
import pytest

import gen
import oracle
import paper_2507_15230_gb300 as gale
from parity_util import assert_bulk_equal, expected_bulk

pytestmark = pytest.mark.gpu

_ORACLE = {}


def _mesh(kind):
    if kind == "grid":
        return gen.small_grid(with_field=False)
    return gen.delaunay_mesh(6000, seed=5, with_field=False)


def _oracle(kind, m):
    if kind not in _ORACLE:
        _ORACLE[kind] = oracle.build_all(m.nv, m.tv, m.seg, m.nclusters)
    return _ORACLE[kind]


@pytest.mark.parametrize("kind", ["grid", "delaunay"])
@pytest.mark.parametrize("team_threads,teams", [(32, 4), (64, 2), (64, 8), (128, 3)])
def test_teams_equal_oracle(kind, team_threads, teams):
    m = _mesh(kind)
    canon, rel = _oracle(kind, m)
    with gale.Context.load(m, device=0) as ctx:
        ctx.set_teams(team_threads, teams)
        bins = ctx.bins()
        tb = [b for b in bins if b["teams"] > 0]
        assert tb, bins
        assert all(b["teams"] == teams and b["threads"] == team_threads for b in tb)
        for _ in range(2):  # the second build replays the captured graph
            ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, np.arange(m.nclusters)))
        rng = np.random.default_rng(team_threads + teams)
        ids = rng.permutation(m.nclusters)[: max(3, m.nclusters // 2)].astype(np.int32)
        for mask in (gale.ALL, gale.VT | gale.TT, gale.VV | gale.ET):
            ctx.build(ids, mask, gale.MODE_BATCHED)
            ctx.synchronize()
            assert_bulk_equal(ctx.export(mask), expected_bulk(rel, canon, ids, mask))
        got = ctx.build_export(ids, gale.ALL, chunks=3)
        assert_bulk_equal(got, expected_bulk(rel, canon, ids))
        ctx.build(ids[:12], gale.ALL, gale.MODE_PER_CLUSTER)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, ids[:12]))
        ctx.set_teams(0, 0)
        assert all(b["teams"] == 0 for b in ctx.bins())
        ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, np.arange(m.nclusters)))


def test_autotune_with_teams_keeps_parity():
    m = _mesh("delaunay")
    canon, rel = _oracle("delaunay", m)
    with gale.Context.load(m, device=0) as ctx:
        ctx.autotune(gale.ALL, reps=1)
        ctx.build(None, gale.ALL, gale.MODE_BATCHED)
        ctx.synchronize()
        assert_bulk_equal(ctx.export(gale.ALL), expected_bulk(rel, canon, np.arange(m.nclusters)))


def test_set_teams_rejects_bad_sizes():
    m = _mesh("grid")
    with gale.Context.load(m, device=0) as ctx:
        for tt, n in [(48, 2), (32, 1), (32, 16), (256, 4), (0, 2)]:
            with pytest.raises(gale.GaleError):
                ctx.set_teams(tt, n)
