"""The generator's on-disk mesh cache (GALE_GEN_CACHE): a cached mesh loads
back bit for bit, other parameters miss the cache, and an unreadable file is
rebuilt."""
import os

import numpy as np

import gen


def same(a, b):
    return (np.array_equal(a.xyz, b.xyz) and np.array_equal(a.tv, b.tv) and np.array_equal(a.seg, b.seg)
            and a.nclusters == b.nclusters and a.name == b.name and a.meta == b.meta
            and ((a.field is None and b.field is None) or np.array_equal(a.field, b.field)))


def test_cache_round_trip_and_misses(tmp_path, monkeypatch):
    fresh = gen.freudenthal_mesh(6, 64, seed=5, jitter=0.2)
    fresh_d = gen.delaunay_mesh(400, seed=9, kd_cap=128, with_field=False)
    monkeypatch.setenv("GALE_GEN_CACHE", str(tmp_path))
    a = gen.freudenthal_mesh(6, 64, seed=5, jitter=0.2)  # built and stored
    files = sorted(os.listdir(tmp_path))
    assert len(files) == 1 and files[0].startswith("freudenthal-")
    b = gen.freudenthal_mesh(6, 64, seed=5, jitter=0.2)  # loaded
    assert same(fresh, a) and same(a, b)
    gen.freudenthal_mesh(6, 64, seed=6, jitter=0.2)  # another seed: another file
    assert len(os.listdir(tmp_path)) == 2
    d1 = gen.delaunay_mesh(400, seed=9, kd_cap=128, with_field=False)
    d2 = gen.delaunay_mesh(400, seed=9, kd_cap=128, with_field=False)
    assert same(fresh_d, d1) and same(d1, d2) and d2.field is None


def test_unreadable_cache_file_is_rebuilt(tmp_path, monkeypatch):
    monkeypatch.setenv("GALE_GEN_CACHE", str(tmp_path))
    a = gen.freudenthal_mesh(4, 32, seed=2)
    (path,) = [os.path.join(tmp_path, f) for f in os.listdir(tmp_path)]
    with open(path, "wb") as f:
        f.write(b"not an npz file")
    b = gen.freudenthal_mesh(4, 32, seed=2)
    assert same(a, b)
    with np.load(path) as z:  # rewritten
        assert "header" in z
