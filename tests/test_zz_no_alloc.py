"""The allocation-free build (gale_build_clusters_noalloc) against the
regular batched build, through the C ABI.

Callers that cannot allocate device memory when they need relations (a
serving thread that must not synchronise the GPU, an application whose own
pool owns all of HBM) own the output arrays and pass them in; the library's
scratch for this call lives in a fixed device array.  The outputs must equal
those of gale_build_clusters bit for bit (integer relations: tolerance
zero), on two calls in a row, since the fixed scratch keeps the previous
call's contents.  This file is collected last."""
import numpy as np
import pytest

import gen
import paper_2507_15230_gb300 as gale

pytestmark = pytest.mark.gpu


def test_noalloc_matches_batched_build_twice():
    import torch
    m = gen.small_grid(with_field=False)
    rng = np.random.default_rng(7)
    lists = [rng.permutation(m.nclusters)[:77].astype(np.int32), np.arange(m.nclusters, dtype=np.int32)[::-1].copy()]
    with gale.Context.load(m, device=0) as ctx:
        for ids in lists:
            ctx.build(ids, gale.ALL, gale.MODE_BATCHED)
            ctx.synchronize()
            want = ctx.export(gale.ALL)
            out = {n: torch.full((max(int(a.size), 1),), -7, dtype=torch.int32, device="cuda") for n, a in want.items()}
            ctx.build_noalloc(ids, gale.ALL, out)
            for n, a in want.items():
                got = out[n][:a.size].cpu().numpy()
                assert np.array_equal(got, a), n


def test_noalloc_rejects_oversized_lists():
    import torch
    m = gen.small_grid(with_field=False)
    with gale.Context.load(m, device=0) as ctx:
        dummy = {n: torch.zeros(1, dtype=torch.int32, device="cuda") for n in gale.ARRAYS}
        with pytest.raises(gale.GaleError) as ei:
            ctx.build_noalloc(np.zeros(4097, np.int32), gale.ALL, dummy)
        assert ei.value.status == 1
        with pytest.raises(gale.GaleError):
            ctx.build_noalloc(np.array([m.nclusters], np.int32), gale.ALL, dummy)
