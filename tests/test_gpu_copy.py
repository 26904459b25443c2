"""gale_copy_to_host: device -> host copies into page-locked and pageable
memory, small (one copy) and large (staged through the context's two
pinned buffers, several chunks with a ragged tail), byte-exact."""
import numpy as np
import pytest

import gen
import paper_2507_15230_gb300 as gale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gale.Context.load(gen.small_grid(), device=0)
    yield c
    c.close()


@pytest.mark.parametrize("n", [0, 1, 1000, (32 << 20) // 4 - 1, (128 << 20) // 4, (5 * (128 << 20)) // 8 + 7])
def test_copy_pageable_matches(ctx, n):
    import torch
    src = torch.randint(-2**31, 2**31 - 1, (max(n, 1),), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    want = src.cpu().numpy()[:n]
    got = ctx.copy_to_host(src.data_ptr(), n)
    assert got.size == n and np.array_equal(got, want)


def test_copy_pinned_and_into_a_given_buffer(ctx):
    import torch
    n = (3 * (128 << 20)) // 4 + 5
    src = torch.arange(n, dtype=torch.int32, device="cuda") * 7 - 3
    torch.cuda.synchronize()
    pinned = torch.empty(n, dtype=torch.int32).pin_memory().numpy()
    got = ctx.copy_to_host(src.data_ptr(), n, out=pinned)
    assert np.array_equal(got, src.cpu().numpy())
    buf = np.full(n + 11, -1, np.int32)  # pageable, larger than the copy
    ctx.copy_to_host(src.data_ptr(), n, out=buf)
    assert np.array_equal(buf[:n], src.cpu().numpy()) and (buf[n:] == -1).all()


def test_copy_repeated_calls_reuse_the_staging_buffers(ctx):
    import torch
    for seed in range(3):
        n = (40 << 20) + seed * 12345
        g = torch.Generator(device="cuda").manual_seed(seed)
        src = torch.randint(0, 1000, (n,), dtype=torch.int32, device="cuda", generator=g)
        torch.cuda.synchronize()
        assert np.array_equal(ctx.copy_to_host(src.data_ptr(), n), src.cpu().numpy())
