"""Consumers of the cluster-relation producer: the lower-link critical-point
classifier (standing in for the paper's CriticalPoints analysis, Section 5.2),
a multi-threaded serving driver, and the discrete gradient (the paper's
DiscreteGradient analysis, Section 5.1) over GPU-built VE, VF and VT.  Built
against the public C ABI only."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgaleconsumers.so")
_SRC = os.path.join(_HERE, "consumers.cpp")
_lib = None


def build(force: bool = False) -> str:
    import paper_2507_15230_gb300 as gale
    gl = gale._build.build()
    os.makedirs(_BUILD, exist_ok=True)
    deps = [_SRC, os.path.join(_ROOT, "include", "gale.h"), gl]
    if not force and os.path.exists(_LIB) and all(os.path.getmtime(d) <= os.path.getmtime(_LIB) for d in deps):
        return _LIB
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC, "-I", os.path.join(_ROOT, "include"),
           "-I", os.path.join(cuda, "include"), "-L", os.path.dirname(gl), "-lgale", "-Wl,-rpath," + os.path.dirname(gl),
           "-L", os.path.join(cuda, "lib64"), "-lcudart", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        import paper_2507_15230_gb300 as gale
        gale.load_library()
        build()
        lib = ctypes.CDLL(_LIB)
        P, i32, i64, u32, u64, f64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.c_double)
        lib.gale_cp_classify.argtypes = [P, P, P, i32, i32, P, P, P, P, P]
        lib.gale_cp_classify.restype = ctypes.c_int
        lib.gale_cp_serve_run.argtypes = [P, P, P, P, P, i32, i32, u32, u64, f64, i32, P, P, P]
        lib.gale_cp_serve_run.restype = ctypes.c_int
        lib.gale_open_loop.argtypes = [P, i32, P, P, P, i64, f64, u64, i32, P, P]
        lib.gale_open_loop.restype = ctypes.c_int
        lib.gale_dg_run.argtypes = [P, P, i64] + [P] * 15 + [i32, i64, P]
        lib.gale_dg_run.restype = ctypes.c_int
        lib.gale_dg_lower_stars.argtypes = [P, P, i64, i64] + [P] * 15
        lib.gale_dg_lower_stars.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def canonical_inputs(field: np.ndarray, vperm: np.ndarray):
    """Field values and input ids in canonical vertex order."""
    vperm = np.ascontiguousarray(vperm, dtype=np.int32)
    return np.ascontiguousarray(field[vperm], dtype=np.float32), vperm


def classify_cluster(f_c, inid_c, rows, v0, vt_off, vt_val, vv_off, vv_val) -> np.ndarray:
    """Critical-point codes of one cluster's vertices from host CSR rows."""
    lib = _load()
    nvo = len(vt_off) - 1
    out = np.empty(max(nvo, 1), np.int8)
    arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in (vt_off, vt_val, vv_off, vv_val)]
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    rc = lib.gale_cp_classify(_p(f_c), _p(inid_c), _p(rows), int(v0), nvo, *[_p(a) if a.size else None for a in arrs],
                              _p(out))
    if rc != 0:
        raise RuntimeError("classifier: link too large")
    return out[:nvo]


def serve_run(ctx, f_c, inid_c, rows, I_V, nthreads=16, mask=15, seed=6, jump_prob=0.1, max_clusters=None,
              null_work=False):
    """Run the serving driver over clusters [0, max_clusters) (all by
    default); returns (codes int8[nv], latencies float64[K],
    dict(wall, requests, d2h_bytes, failures, copy_s, integrate_s)).
    null_work: each view is released as soon as it is served (no copy, no
    classification; the codes stay -9), to measure the producer alone."""
    lib = _load()
    K = len(I_V) - 1
    if max_clusters is not None:
        K = min(K, int(max_clusters))
    cls = np.full(len(f_c), -9, np.int8)
    lat = np.zeros(K, np.float64)
    st = np.zeros(6, np.float64)
    I_V = np.ascontiguousarray(I_V, dtype=np.int64)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    lib.gale_cp_serve_run(ctx._h, _p(f_c), _p(inid_c), _p(rows), _p(I_V), K, nthreads, mask, seed, jump_prob,
                          1 if null_work else 0, _p(cls), _p(lat), _p(st))
    return cls, lat, {"wall": st[0], "requests": int(st[1]), "d2h_bytes": int(st[2]), "failures": int(st[3]),
                      "copy_s": float(st[4]), "integrate_s": float(st[5])}


def open_loop(ctxs, mi, ks, masks, rate=None, seed=0, workers=64):
    """Native open-loop driver (gale_open_loop): Poisson arrivals at `rate`
    requests/s (None: all at once, a capacity run) of (mesh mi[i], cluster
    ks[i], mask masks[i]); returns (latency seconds per request, wall
    seconds, failures, first failing request or -1)."""
    lib = _load()
    n = len(mi)
    handles = (ctypes.c_void_p * len(ctxs))(*[c._h for c in ctxs])
    mi = np.ascontiguousarray(mi, dtype=np.int32)
    ks = np.ascontiguousarray(ks, dtype=np.int32)
    masks = np.ascontiguousarray(masks, dtype=np.uint32)
    lat = np.zeros(n, np.float64)
    st = np.zeros(3, np.float64)
    rc = lib.gale_open_loop(ctypes.cast(handles, ctypes.c_void_p), len(ctxs), _p(mi), _p(ks), _p(masks), n,
                            float(rate) if rate else 0.0, int(seed), int(workers), _p(lat), _p(st))
    if rc != 0:
        raise RuntimeError("gale_open_loop failed")
    return lat, float(st[0]), int(st[1]), int(st[2])


def csr_from_bulk(off_b, val_b, I_V):
    """Whole-mesh CSR (int64 offsets, rows in canonical vertex order) from a
    bulk array pair laid out cluster after cluster, each cluster's offsets
    (own vertices + 1) starting at 0."""
    I_V = np.asarray(I_V, dtype=np.int64)
    nvo = np.diff(I_V)
    starts = np.concatenate([[0], np.cumsum(nvo + 1)[:-1]]).astype(np.int64)
    counts = off_b[starts + nvo].astype(np.int64)
    vbase = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    keep = np.ones(off_b.size, bool)
    keep[starts + nvo] = False
    off = off_b[keep].astype(np.int64) + np.repeat(vbase, nvo)
    return np.concatenate([off, [int(counts.sum())]]).astype(np.int64), np.ascontiguousarray(val_b, dtype=np.int32)


def discrete_gradient_arrays(f_c, inid_c, ve, vf, vt, ev, fv, tv, nthreads=16, grain=1024):
    """gale_dg_run on host arrays: ve, vf, vt are (offsets, values) CSR pairs
    indexed by canonical vertex; ev, fv, tv the vertex lists (consumers.cpp).
    Returns (dict v_up, e_down, e_up, f_down, f_up, t_down; wall seconds)."""
    lib = _load()
    nv = len(f_c)
    nE, nF, nT = np.asarray(ev).size // 2, np.asarray(fv).size // 3, np.asarray(tv).size // 4
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32).reshape(-1)
    i64 = lambda a: np.ascontiguousarray(a, dtype=np.int64)
    rel = [i64(ve[0]), i32(ve[1]), i64(vf[0]), i32(vf[1]), i64(vt[0]), i32(vt[1]), i32(ev), i32(fv), i32(tv)]
    out = {"v_up": np.empty(nv, np.int32), "e_down": np.empty(nE, np.int32), "e_up": np.empty(nE, np.int32),
           "f_down": np.empty(nF, np.int32), "f_up": np.empty(nF, np.int32), "t_down": np.empty(nT, np.int32)}
    st = np.zeros(2, np.float64)
    ptr = lambda a: a.ctypes.data if a.size else None
    f_c = np.ascontiguousarray(f_c, dtype=np.float32)
    inid_c = np.ascontiguousarray(inid_c, dtype=np.int32)
    rc = lib.gale_dg_run(_p(f_c), _p(inid_c), nv, *[ptr(a) for a in rel], *[ptr(a) for a in out.values()],
                         int(nthreads), int(grain), _p(st))
    if rc == -2:
        raise MemoryError("discrete gradient: the vertex key array cannot be allocated")
    if rc != 0:
        raise RuntimeError("discrete gradient: inconsistent relations")
    return out, float(st[0])


def lower_stars_into(out, f_c, inid_c, v_begin, v_end, ve, vf, vt, ev, fv, tv):
    """gale_dg_lower_stars: the lower stars of vertices [v_begin, v_end) on
    the calling thread, written into `out` (the dict discrete_gradient_arrays
    returns: every simplex whose highest vertex is in the range gets both
    of its entries)."""
    lib = _load()
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32).reshape(-1)
    i64 = lambda a: np.ascontiguousarray(a, dtype=np.int64)
    rel = [i64(ve[0]), i32(ve[1]), i64(vf[0]), i32(vf[1]), i64(vt[0]), i32(vt[1]), i32(ev), i32(fv), i32(tv)]
    ptr = lambda a: a.ctypes.data if a.size else None
    f_c = np.ascontiguousarray(f_c, dtype=np.float32)
    inid_c = np.ascontiguousarray(inid_c, dtype=np.int32)
    names = ("v_up", "e_down", "e_up", "f_down", "f_up", "t_down")
    assert all(out[k].dtype == np.int32 and out[k].flags["C_CONTIGUOUS"] for k in names)
    rc = lib.gale_dg_lower_stars(_p(f_c), _p(inid_c), int(v_begin), int(v_end), *[ptr(a) for a in rel],
                                 *[ptr(out[k]) for k in names])
    if rc != 0:
        raise RuntimeError("discrete gradient: inconsistent relations")
    return out


def gather_gradient_relations(ctx, order=None):
    """The relations the discrete gradient reads, from a loaded context:
    the enumeration (gale_enumerate), VE and VF from the GPU coboundary pass,
    VT from a batched build, and TV.  (FE and TF are looked up by the
    consumer itself.)  Returns a dict of host arrays."""
    import paper_2507_15230_gb300 as gale
    en = ctx.enumerate(order) if order is not None else None
    cb = ctx.coboundary(gale.CB_VE | gale.CB_VF)
    if en is None:
        en = ctx.enumeration()
    I_V, _, _ = ctx.intervals()
    ctx.build(None, gale.VT, gale.MODE_BATCHED)
    ctx.synchronize()
    b = ctx.export(gale.VT)
    vt = csr_from_bulk(b["vt_off"], b["vt_val"], I_V)
    rows = ctx.rows()
    return {"ve": cb["VE"], "vf": cb["VF"], "vt": vt, "ev": en["E"], "fv": en["F"], "tv": rows}


def discrete_gradient(ctx, f_c, inid_c, rel=None, nthreads=16, order=None):
    """The discrete gradient of a field on a loaded context (relations
    gathered with gather_gradient_relations unless given)."""
    if rel is None:
        rel = gather_gradient_relations(ctx, order)
    return discrete_gradient_arrays(f_c, inid_c, rel["ve"], rel["vf"], rel["vt"], rel["ev"], rel["fv"], rel["tv"],
                                    nthreads=nthreads)
