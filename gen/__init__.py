"""Seeded synthetic inputs: meshes, kd-tree vertex partitions and scalar fields.

Both the CPU oracle and the CUDA path consume what this module produces; it
holds none of the relation arithmetic.  The workloads stand in for the paper's
datasets (Section 5.1, Table 2), which are not available here:

* ``freudenthal_mesh`` - an n^3 cube grid, 6 tets per cube (Kuhn/Freudenthal),
  vertex ids permuted from a seed, optional coordinate jitter.  At n = 256 it
  has 16.97M vertices / 100.7M tets, the shape of the paper's Stent mesh.
* ``delaunay_mesh`` - Delaunay tetrahedralisation of a seeded Gaussian-mixture
  point cloud, standing in for the unstructured Fish / Hole meshes.
* ``kdtree_partition`` - the vertex segmentation the method needs as input
  (Section 4.3 "Input data"); a kd-tree replaces the paper's PR octree.
* ``gaussian_field`` - a float32 scalar field (sum of Gaussians) for the
  critical-point consumer.

Generated meshes can be kept on disk so that 100M-tet inputs are not rebuilt
on every run: with ``GALE_GEN_CACHE`` set to a directory, ``freudenthal_mesh``
and ``delaunay_mesh`` store each mesh as ``.npz`` arrays plus a JSON header of
the generator's parameters, and load it back when every parameter matches.
A file that cannot be read or whose header differs is rebuilt.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
import subprocess
from dataclasses import dataclass, field as dc_field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgalegen.so")
_SRCS = ["gen.c", "gen_delaunay.c"]

_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library with gcc (portable C, no -march)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SRCS if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(_LIB):
        lib_m = os.path.getmtime(_LIB)
        if all(os.path.getmtime(s) <= lib_m for s in srcs):
            return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.gen_freudenthal.argtypes = [i32, i32, f64, u64, P, P]
        lib.gen_freudenthal.restype = ctypes.c_int
        lib.gen_kdtree.argtypes = [i64, P, i32, i32, i32, i32, u64, P]
        lib.gen_kdtree.restype = i32
        lib.gen_field.argtypes = [i64, P, i32, P, P, u64, P]
        lib.gen_field.restype = ctypes.c_int
        lib.gen_points.argtypes = [i64, f64, i32, f64, f64, i32, u64, P]
        lib.gen_points.restype = ctypes.c_int
        lib.gen_permutation.argtypes = [i64, u64, P]
        lib.gen_permutation.restype = ctypes.c_int
        if hasattr(lib, "gen_delaunay"):
            lib.gen_delaunay.argtypes = [i64, P, P, ctypes.POINTER(i64)]
            lib.gen_delaunay.restype = ctypes.c_int
            lib.gen_delaunay_fetch.argtypes = [P]
            lib.gen_delaunay_fetch.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


@dataclass
class Mesh:
    """A tetrahedral mesh with a vertex partition, in the paper's input form
    (Section 4.3): coordinates V, tetrahedra T (4 vertex ids each, the TV
    relation) and segment ids S per vertex."""

    xyz: np.ndarray  # float32 [nv, 3]
    tv: np.ndarray  # int32 [nt, 4]
    seg: np.ndarray  # int32 [nv]
    nclusters: int
    field: np.ndarray | None = None  # float32 [nv]
    name: str = ""
    meta: dict = dc_field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tv.shape[0])


def freudenthal_grid(n: int, permute: bool = True, jitter: float = 0.0, seed: int = 1):
    """(xyz float32[V,3], tv int32[T,4]) of the Freudenthal subdivision of an n^3 grid."""
    lib = _load()
    nv, nt = (n + 1) ** 3, 6 * n ** 3
    xyz = np.empty((nv, 3), dtype=np.float32)
    tv = np.empty((nt, 4), dtype=np.int32)
    rc = lib.gen_freudenthal(n, 1 if permute else 0, float(jitter), seed, _ptr(xyz), _ptr(tv))
    if rc != 0:
        raise ValueError(f"gen_freudenthal failed for n={n}")
    return xyz, tv


def kdtree_partition(xyz: np.ndarray, cap: int, uneven: bool = False, min_leaf: int = 64, min_cap: int = 32,
                     seed: int = 0):
    """(seg int32[nv], nleaves): kd-tree leaves of at most ``cap`` vertices
    (uneven: per-node caps log-uniform in [min_cap, cap], nodes below
    ``min_leaf`` always stop)."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    seg = np.empty(xyz.shape[0], dtype=np.int32)
    k = lib.gen_kdtree(xyz.shape[0], _ptr(xyz), cap, 1 if uneven else 0, min_leaf, min_cap, seed, _ptr(seg))
    if k < 0:
        raise ValueError("gen_kdtree failed")
    return seg, int(k)


def gaussian_field(xyz: np.ndarray, ngauss: int, lo, hi, seed: int) -> np.ndarray:
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    f = np.empty(xyz.shape[0], dtype=np.float32)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    if lib.gen_field(xyz.shape[0], _ptr(xyz), ngauss, _ptr(lo), _ptr(hi), seed, _ptr(f)) != 0:
        raise ValueError("gen_field failed")
    return f


def permutation(n: int, seed: int) -> np.ndarray:
    lib = _load()
    p = np.empty(n, dtype=np.int32)
    if lib.gen_permutation(n, seed, _ptr(p)) != 0:
        raise ValueError("gen_permutation failed")
    return p


_CACHE_FORMAT = 1


def _cache_path(params: dict):
    d = os.environ.get("GALE_GEN_CACHE")
    if not d:
        return None
    key = hashlib.sha1(json.dumps(params, sort_keys=True).encode()).hexdigest()[:20]
    return os.path.join(d, f"{params['kind']}-{key}.npz")


def _cached(params: dict, make):
    """make() -> Mesh, through the on-disk cache when GALE_GEN_CACHE is set."""
    path = _cache_path(params)
    if path and os.path.exists(path):
        try:
            with np.load(path, allow_pickle=False) as z:
                head = json.loads(str(z["header"]))
                if head.get("format") == _CACHE_FORMAT and head.get("params") == params:
                    f = z["field"] if bool(head["has_field"]) else None
                    return Mesh(z["xyz"], z["tv"], z["seg"], int(head["nclusters"]), f, head["name"],
                                head["meta"])
        except Exception:
            pass  # unreadable or stale: rebuilt below
    m = make()
    if path:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        head = {"format": _CACHE_FORMAT, "params": params, "nclusters": m.nclusters, "name": m.name,
                "meta": m.meta, "has_field": m.field is not None}
        tmp = f"{path}.tmp{os.getpid()}.npz"
        np.savez(tmp, xyz=m.xyz, tv=m.tv, seg=m.seg,
                 field=m.field if m.field is not None else np.zeros(0, np.float32),
                 header=np.array(json.dumps(head)))
        os.replace(tmp, path)
    return m


def freudenthal_mesh(n: int, kd_cap: int, seed: int = 1, field_seed: int = 2, jitter: float = 0.0,
                     ngauss: int = 4, with_field: bool = True, name: str = "") -> Mesh:
    """Freudenthal grid, permuted ids, kd-tree leaves of <= kd_cap vertices,
    sum-of-Gaussians field.  The small workload is n=16, cap 64; the
    at-scale workload n=256, jitter 0.3, cap 512."""
    params = {"kind": "freudenthal", "n": n, "kd_cap": kd_cap, "seed": seed, "field_seed": field_seed,
              "jitter": jitter, "ngauss": ngauss, "with_field": with_field, "name": name}
    return _cached(params, lambda: _freudenthal_mesh(n, kd_cap, seed, field_seed, jitter, ngauss, with_field,
                                                     name))


def _freudenthal_mesh(n, kd_cap, seed, field_seed, jitter, ngauss, with_field, name) -> Mesh:
    xyz, tv = freudenthal_grid(n, True, jitter, seed)
    seg, k = kdtree_partition(xyz, kd_cap)
    f = gaussian_field(xyz, ngauss, [0, 0, 0], [n, n, n], field_seed) if with_field else None
    return Mesh(xyz, tv, seg, k, f, name or f"freudenthal{n}^3/kd{kd_cap}",
                {"kind": "freudenthal", "n": n, "kd_cap": kd_cap, "seed": seed, "jitter": jitter})


def delaunay_points(npts: int, seed: int, frac_mix: float = 0.7, nmix: int = 8, smin: float = 0.03,
                    smax: float = 0.08, bits: int = 20) -> np.ndarray:
    """Unique int64 grid points [m, 3] (snapped to a 2^bits grid, duplicates
    removed, order as drawn) from a Gaussian mixture plus uniform background."""
    lib = _load()
    pts = np.empty((npts, 3), dtype=np.int64)
    if lib.gen_points(npts, frac_mix, nmix, smin, smax, bits, seed, _ptr(pts)) != 0:
        raise ValueError("gen_points failed")
    _, first = np.unique(pts, axis=0, return_index=True)
    return np.ascontiguousarray(pts[np.sort(first)])


def delaunay_tets(pts: np.ndarray) -> np.ndarray:
    """Delaunay tetrahedralisation (Bowyer-Watson with exact integer
    predicates) of integer points; int32 [nt, 4] of point indices."""
    lib = _load()
    if not hasattr(lib, "gen_delaunay"):
        raise RuntimeError("Delaunay generator not built")
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    nt = ctypes.c_int64(0)
    h = ctypes.c_void_p(0)
    rc = lib.gen_delaunay(pts.shape[0], _ptr(pts), ctypes.byref(h), ctypes.byref(nt))
    if rc != 0:
        raise RuntimeError(f"gen_delaunay failed ({rc})")
    tv = np.empty((nt.value, 4), dtype=np.int32)
    lib.gen_delaunay_fetch(_ptr(tv))
    return tv


def delaunay_mesh(npts: int, seed: int, kd_cap: int = 2048, uneven: bool = True, min_leaf: int = 64,
                  min_cap: int = 32, bits: int = 20, ngauss_field: int = 4, with_field: bool = True,
                  name: str = "") -> Mesh:
    """Delaunay mesh of a Gaussian-mixture point cloud with an uneven kd-tree
    partition (leaves of 32 .. 2048 vertices)."""
    params = {"kind": "delaunay", "npts": npts, "seed": seed, "kd_cap": kd_cap, "uneven": uneven,
              "min_leaf": min_leaf, "min_cap": min_cap, "bits": bits, "ngauss_field": ngauss_field,
              "with_field": with_field, "name": name}
    return _cached(params, lambda: _delaunay_mesh(npts, seed, kd_cap, uneven, min_leaf, min_cap, bits,
                                                  ngauss_field, with_field, name))


def _delaunay_mesh(npts, seed, kd_cap, uneven, min_leaf, min_cap, bits, ngauss_field, with_field, name) -> Mesh:
    pts = delaunay_points(npts, seed, bits=bits)
    tv = delaunay_tets(pts)
    xyz = (pts.astype(np.float64) / float(1 << bits)).astype(np.float32)
    seg, k = kdtree_partition(xyz, kd_cap, uneven=uneven, min_leaf=min_leaf, min_cap=min_cap, seed=seed)
    f = gaussian_field(xyz, ngauss_field, [0, 0, 0], [1, 1, 1], seed + 1000) if with_field else None
    return Mesh(xyz, tv, seg, k, f, name or f"delaunay{npts}/kd{min_cap}-{kd_cap}",
                {"kind": "delaunay", "npts": npts, "seed": seed, "kd_cap": kd_cap, "uneven": uneven})


# Named workloads (sizes and seeds of each synthetic configuration).
def small_grid(with_field: bool = True) -> Mesh:
    """16^3 Freudenthal grid, 4,913 vertices / 24,576 tets, permuted ids (seed 1),
    kd leaves <= 64 vertices, field = sum of 4 Gaussians (seed 2)."""
    return freudenthal_mesh(16, 64, seed=1, field_seed=2, jitter=0.0, ngauss=4, with_field=with_field,
                            name="grid16^3-kd64")


def scale_grid(n: int = 256, with_field: bool = False, ngauss: int = 16) -> Mesh:
    """256^3 Freudenthal grid, 16.97M vertices / 100.7M tets, jitter +-0.3 cell
    (seed 3), permuted ids, kd leaves <= 512 vertices, field seed 4."""
    return freudenthal_mesh(n, 512, seed=3, field_seed=4, jitter=0.3, ngauss=ngauss, with_field=with_field,
                            name=f"grid{n}^3-jitter0.3-kd512")
