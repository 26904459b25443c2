"""CPU oracle for the cluster-relation producer (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product never imports
this package; it shares no code with the CUDA path.

The arithmetic lives in ``oracle.c`` (plain C, every function cites the
passage it follows).  This module compiles it with gcc and wraps it:

* ``validate``              - input checks (Section 4.3, "Input data")
* ``canonicalize``          - canonical vertex / tet numbering, interval arrays
                              I_V, I_T, internal rule (Section 4.3)
* ``relations``             - VT, VV, ET, TT of the whole mesh (Section 2.2,
                              Table 1), global formulation
* ``cluster_relations``     - the same for one cluster, by rescanning the mesh
* ``working_set``           - T_ex (Section 4.3, "Initialization") and the
                              face halo of one cluster
* ``cluster_view``          - slices a global result into one cluster's
                              self-contained CSR (offsets starting at 0)
* ``enumerate_simplices``   - edge / triangle enumeration E, F, I_E, I_F
                              (Section 4.3, "Initialization"), plain Python
* ``boundary``              - FE, TE, TF by lookup (Section 4.4)
* ``coboundary``            - VE, VF, EF, FT of the whole mesh (Table 1)
* ``lower_star_gradient``   - the discrete gradient of a vertex field
                              (Section 5.1, DiscreteGradient), plain Python
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

OK, EINVAL, ENOMEM = 0, 1, 2
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c (plain C, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Rel(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("nt", ctypes.c_int64), ("ne", ctypes.c_int64),
                ("vt_off", ctypes.POINTER(ctypes.c_int64)), ("vt_val", ctypes.POINTER(ctypes.c_int32)),
                ("vv_off", ctypes.POINTER(ctypes.c_int64)), ("vv_val", ctypes.POINTER(ctypes.c_int32)),
                ("eu_off", ctypes.POINTER(ctypes.c_int64)), ("e_w", ctypes.POINTER(ctypes.c_int32)),
                ("et_off", ctypes.POINTER(ctypes.c_int64)), ("et_val", ctypes.POINTER(ctypes.c_int32)),
                ("tt_off", ctypes.POINTER(ctypes.c_int64)), ("tt_val", ctypes.POINTER(ctypes.c_int32))]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.oracle_validate.argtypes = [i64, i64, P, P, i32]
        lib.oracle_canon_vertices.argtypes = [i64, P, i32, P, P, P]
        lib.oracle_canon_tets.argtypes = [i64, P, P, P, P, i32, P, P, P]
        lib.oracle_relations.argtypes = [i64, i64, P, ctypes.POINTER(_Rel)]
        lib.oracle_cluster_relations.argtypes = [i64, i64, P, P, P, i32, ctypes.POINTER(_Rel)]
        lib.oracle_working_set.argtypes = [i64, i64, P, P, P, i32, P, ctypes.POINTER(i64), P, ctypes.POINTER(i64)]
        lib.oracle_localized_build.argtypes = [i64, i64, P, P, P, i32, i32, P, P, P]
        lib.oracle_localized_cluster.argtypes = [i64, i64, P, P, P, i32, i32, ctypes.POINTER(_Rel)]
        lib.oracle_rel_free.argtypes = [ctypes.POINTER(_Rel)]
        lib.oracle_rel_free.restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def validate(nv: int, tv: np.ndarray, seg: np.ndarray, nclusters: int) -> int:
    tv = np.ascontiguousarray(tv, dtype=np.int32).reshape(-1, 4)
    seg = np.ascontiguousarray(seg, dtype=np.int32)
    if seg.shape[0] != nv:
        return EINVAL
    return _load().oracle_validate(nv, tv.shape[0], _p(tv), _p(seg), nclusters)


def canonicalize(nv: int, tv: np.ndarray, seg: np.ndarray, nclusters: int) -> dict:
    """Canonical numbering.  Returns cid (input -> canonical vertex), vperm
    (canonical -> input), I_V [K+1], rows [T,4] (canonical, ascending, in
    canonical tet order), tperm (canonical -> input tet), I_T [K+1]."""
    lib = _load()
    tv = np.ascontiguousarray(tv, dtype=np.int32).reshape(-1, 4)
    seg = np.ascontiguousarray(seg, dtype=np.int32)
    nt = tv.shape[0]
    cid = np.empty(nv, np.int32)
    vperm = np.empty(nv, np.int32)
    I_V = np.empty(nclusters + 1, np.int64)
    if lib.oracle_canon_vertices(nv, _p(seg), nclusters, _p(cid), _p(vperm), _p(I_V)) != OK:
        raise MemoryError("oracle_canon_vertices")
    rows = np.empty((nt, 4), np.int32)
    tperm = np.empty(nt, np.int32)
    I_T = np.empty(nclusters + 1, np.int64)
    if lib.oracle_canon_tets(nt, _p(tv), _p(cid), _p(vperm), _p(seg), nclusters, _p(rows), _p(tperm), _p(I_T)) != OK:
        raise MemoryError("oracle_canon_tets")
    return {"nv": nv, "nt": nt, "K": nclusters, "cid": cid, "vperm": vperm, "I_V": I_V, "rows": rows,
            "tperm": tperm, "I_T": I_T}


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def _unpack(r: _Rel, nrows_v: int, nrows_t: int) -> dict:
    vt_off = _arr(r.vt_off, nrows_v + 1, np.int64)
    vv_off = _arr(r.vv_off, nrows_v + 1, np.int64)
    eu_off = _arr(r.eu_off, nrows_v + 1, np.int64)
    ne = int(r.ne)
    et_off = _arr(r.et_off, ne + 1, np.int64)
    tt_off = _arr(r.tt_off, nrows_t + 1, np.int64)
    return {
        "vt_off": vt_off, "vt_val": _arr(r.vt_val, int(vt_off[-1]), np.int32),
        "vv_off": vv_off, "vv_val": _arr(r.vv_val, int(vv_off[-1]), np.int32),
        "eu_off": eu_off, "e_w": _arr(r.e_w, ne, np.int32),
        "et_off": et_off, "et_val": _arr(r.et_val, int(et_off[-1]), np.int32),
        "tt_off": tt_off, "tt_val": _arr(r.tt_val, int(tt_off[-1]), np.int32),
        "ne": ne,
    }


def relations(canon: dict) -> dict:
    """VT, VV, ET, TT of the whole mesh (global CSR, canonical ids)."""
    lib = _load()
    r = _Rel()
    rows = np.ascontiguousarray(canon["rows"])
    if lib.oracle_relations(canon["nv"], canon["nt"], _p(rows), ctypes.byref(r)) != OK:
        raise MemoryError("oracle_relations")
    try:
        return _unpack(r, canon["nv"], canon["nt"])
    finally:
        lib.oracle_rel_free(ctypes.byref(r))


def cluster_relations(canon: dict, k: int) -> dict:
    """VT/VV/ET rows of cluster k's vertices and TT rows of its internal tets,
    found by rescanning the whole mesh; offsets start at 0."""
    lib = _load()
    r = _Rel()
    rows = np.ascontiguousarray(canon["rows"])
    I_V, I_T = canon["I_V"], canon["I_T"]
    if lib.oracle_cluster_relations(canon["nv"], canon["nt"], _p(rows), _p(I_V), _p(I_T), k, ctypes.byref(r)) != OK:
        raise MemoryError("oracle_cluster_relations")
    try:
        return _unpack(r, int(I_V[k + 1] - I_V[k]), int(I_T[k + 1] - I_T[k]))
    finally:
        lib.oracle_rel_free(ctypes.byref(r))


def localized_build(canon: dict, nthreads: int = 1, digests: bool = True):
    """Per-cluster localized producer: every cluster's working set (T_k and
    its face halo) gathered once, then VT, VV, ET and TT of each cluster
    built from its working set alone, nthreads threads over the clusters.
    Returns (sizes int64[K, 5] as cluster_sizes gives them, digests uint64[K]
    as relation_digest gives them (or None), (init seconds, build seconds))."""
    lib = _load()
    rows = np.ascontiguousarray(canon["rows"])
    K = int(canon["K"])
    sizes = np.zeros((K, 5), np.int64)
    dig = np.zeros(K, np.uint64) if digests else None
    sec = np.zeros(2, np.float64)
    rc = lib.oracle_localized_build(canon["nv"], canon["nt"], _p(rows), _p(canon["I_V"]), _p(canon["I_T"]), K,
                                    int(nthreads), _p(sizes), _p(dig) if digests else None, _p(sec))
    if rc != OK:
        raise RuntimeError(f"oracle_localized_build: status {rc}")
    return sizes, dig, (float(sec[0]), float(sec[1]))


def localized_cluster(canon: dict, k: int) -> dict:
    """Cluster k's relations by the localized producer (offsets start at 0),
    in the layout of cluster_relations."""
    lib = _load()
    r = _Rel()
    rows = np.ascontiguousarray(canon["rows"])
    I_V, I_T = canon["I_V"], canon["I_T"]
    if lib.oracle_localized_cluster(canon["nv"], canon["nt"], _p(rows), _p(I_V), _p(I_T), int(canon["K"]), k,
                                    ctypes.byref(r)) != OK:
        raise RuntimeError("oracle_localized_cluster")
    try:
        return _unpack(r, int(I_V[k + 1] - I_V[k]), int(I_T[k + 1] - I_T[k]))
    finally:
        lib.oracle_rel_free(ctypes.byref(r))


_DIGEST_P = (1000003, 1000033, 1000037, 1000039, 1000081, 1000099, 1000117, 1000121, 1000133, 1000151)
_DIGEST_KEYS = ("vt_off", "vt_val", "vv_off", "vv_val", "eu_off", "e_w", "et_off", "et_val", "tt_off", "tt_val")


def relation_digest(v: dict) -> int:
    """Order-sensitive digest of one cluster's ten arrays (the definition the
    localized producer uses): for array a of length n, P_a (n + 1) plus the
    sum over i of (x_i + 7)(i + 1) P_a, modulo 2^64."""
    d = 0
    for key, p in zip(_DIGEST_KEYS, _DIGEST_P):
        x = np.asarray(v[key]).astype(np.int64).astype(np.uint64)
        n = x.size
        i = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            d += int((((x + np.uint64(7)) * i) * np.uint64(p)).sum(dtype=np.uint64)) + p * (n + 1)
    return d % (1 << 64)


def working_set(canon: dict, k: int):
    """(T_ex(k), halo(k)) as ascending canonical tet ids."""
    lib = _load()
    nt = canon["nt"]
    ext = np.empty(max(nt, 1), np.int32)
    halo = np.empty(max(nt, 1), np.int32)
    ne, nh = ctypes.c_int64(0), ctypes.c_int64(0)
    rows = np.ascontiguousarray(canon["rows"])
    lib.oracle_working_set(canon["nv"], nt, _p(rows), _p(canon["I_V"]), _p(canon["I_T"]), k, _p(ext),
                           ctypes.byref(ne), _p(halo), ctypes.byref(nh))
    return ext[:ne.value].copy(), halo[:nh.value].copy()


def cluster_view(rel: dict, canon: dict, k: int) -> dict:
    """Cluster k's slice of a global result, as a self-contained CSR: VT/VV
    rows for its vertices, ET edges whose lower endpoint it owns (eu_off per
    vertex, e_w, et_off per edge), TT rows for its internal tets; every offset
    array starts at 0."""
    v0, v1 = int(canon["I_V"][k]), int(canon["I_V"][k + 1])
    t0, t1 = int(canon["I_T"][k]), int(canon["I_T"][k + 1])

    def sl(off, val, a, b):
        o = off[a:b + 1]
        return (o - o[0]).astype(np.int64), val[o[0]:o[-1]]

    vt_off, vt_val = sl(rel["vt_off"], rel["vt_val"], v0, v1)
    vv_off, vv_val = sl(rel["vv_off"], rel["vv_val"], v0, v1)
    eu = rel["eu_off"][v0:v1 + 1]
    e0, e1 = int(eu[0]), int(eu[-1])
    et_off, et_val = sl(rel["et_off"], rel["et_val"], e0, e1)
    tt_off, tt_val = sl(rel["tt_off"], rel["tt_val"], t0, t1)
    return {"vt_off": vt_off, "vt_val": vt_val, "vv_off": vv_off, "vv_val": vv_val,
            "eu_off": (eu - e0).astype(np.int64), "e_w": rel["e_w"][e0:e1], "et_off": et_off, "et_val": et_val,
            "tt_off": tt_off, "tt_val": tt_val, "ne": e1 - e0}


def cluster_sizes(rel: dict, canon: dict) -> np.ndarray:
    """int64 [K, 5]: per cluster |VT|, |VV|, #edges, |ET|, |TT| (entries)."""
    I_V, I_T = canon["I_V"], canon["I_T"]
    vt = rel["vt_off"][I_V[1:]] - rel["vt_off"][I_V[:-1]]
    vv = rel["vv_off"][I_V[1:]] - rel["vv_off"][I_V[:-1]]
    e = rel["eu_off"][I_V[1:]] - rel["eu_off"][I_V[:-1]]
    et = rel["et_off"][rel["eu_off"][I_V[1:]]] - rel["et_off"][rel["eu_off"][I_V[:-1]]]
    tt = rel["tt_off"][I_T[1:]] - rel["tt_off"][I_T[:-1]]
    return np.stack([vt, vv, e, et, tt], axis=1).astype(np.int64)


def build_all(nv: int, tv: np.ndarray, seg: np.ndarray, nclusters: int):
    """The whole oracle pipeline (validate, canonicalize, relations); the
    unit the CPU baseline times."""
    rc = validate(nv, tv, seg, nclusters)
    if rc != OK:
        raise ValueError(f"oracle_validate: {rc}")
    canon = canonicalize(nv, tv, seg, nclusters)
    return canon, relations(canon)


# ---------------------------------------------------------------------------
# Edge and triangle enumeration and boundary relations (Section 4.3
# "Initialization": E and F are enumerated on the CPU by iterating the
# tetrahedra of each segment, all two- and three-vertex combinations, with
# interval arrays I_E, I_F; Section 4.4: a consumer computes a boundary
# relation such as FE by looking the combinations up in E within the owning
# segment's interval).  An edge or triangle belongs to the segment of its
# lowest vertex (the internal rule).  Two numberings:
#   "sorted" - within each segment, lexicographic in canonical ids;
#   "first"  - within each segment, in order of first appearance while the
#              tetrahedra are visited in canonical order, each tetrahedron's
#              combinations in combination order (the numbering of the
#              worked example FE(f5) = {e2, e6, e9}).
# Plain Python over the canonical rows; meant for small meshes.
# ---------------------------------------------------------------------------

def enumerate_simplices(canon: dict, order: str = "sorted") -> dict:
    """E (list of (u, w)), F (list of (a, b, c)), I_E, I_F (length K+1)."""
    if order not in ("sorted", "first"):
        raise ValueError("order is 'sorted' or 'first'")
    rows = canon["rows"]
    I_V = np.asarray(canon["I_V"])
    K = I_V.size - 1

    def seg(v):
        return int(np.searchsorted(I_V, v, side="right") - 1)

    per_e = [[] for _ in range(K)]
    per_f = [[] for _ in range(K)]
    seen_e, seen_f = set(), set()
    for t in range(rows.shape[0]):
        r = [int(x) for x in rows[t]]  # ascending
        for i in range(4):
            for j in range(i + 1, 4):
                e = (r[i], r[j])
                if e not in seen_e:
                    seen_e.add(e)
                    per_e[seg(e[0])].append(e)
        for i in range(4):
            for j in range(i + 1, 4):
                for k in range(j + 1, 4):
                    f = (r[i], r[j], r[k])
                    if f not in seen_f:
                        seen_f.add(f)
                        per_f[seg(f[0])].append(f)
    if order == "sorted":
        per_e = [sorted(x) for x in per_e]
        per_f = [sorted(x) for x in per_f]
    E = [e for x in per_e for e in x]
    F = [f for x in per_f for f in x]
    I_E = [0]
    for x in per_e:
        I_E.append(I_E[-1] + len(x))
    I_F = [0]
    for x in per_f:
        I_F.append(I_F[-1] + len(x))
    return {"E": E, "F": F, "I_E": I_E, "I_F": I_F}


def boundary(canon: dict, enum: dict, relation: str, ids) -> list:
    """Boundary relations by lookup (Section 4.4): "FE" - a triangle's edges
    (a,b), (a,c), (b,c); "TE" - a tetrahedron's six edges in combination
    order; "TF" - a tetrahedron's four triangles (a,b,c), (a,b,d), (a,c,d),
    (b,c,d).  Ids are global edge / triangle ids of `enum`."""
    eid = {e: i for i, e in enumerate(enum["E"])}
    fid = {f: i for i, f in enumerate(enum["F"])}
    rows = canon["rows"]
    out = []
    for s in ids:
        if relation == "FE":
            a, b, c = enum["F"][int(s)]
            out.append([eid[(a, b)], eid[(a, c)], eid[(b, c)]])
        elif relation == "TE":
            r = [int(x) for x in rows[int(s)]]
            out.append([eid[(r[i], r[j])] for i in range(4) for j in range(i + 1, 4)])
        elif relation == "TF":
            r = [int(x) for x in rows[int(s)]]
            out.append([fid[(r[i], r[j], r[k])] for i in range(4) for j in range(i + 1, 4) for k in range(j + 1, 4)])
        else:
            raise ValueError("relation is 'FE', 'TE' or 'TF'")
    return out


def coboundary(canon: dict, enum: dict) -> dict:
    """Coboundary relations of the whole mesh in the ids of `enum` (the
    relations Section 4.6 computes per segment on the GPU: VE, VF, EF, FT,
    Section 5 / Table 1), each row sorted ascending:
      VE[v] - edges containing vertex v;   VF[v] - triangles containing v;
      EF[e] - triangles containing edge e; FT[f] - tets containing triangle f.
    Lists of lists, rows in vertex / edge id / triangle id order."""
    nv = int(canon["nv"])
    rows = canon["rows"]
    E, F = enum["E"], enum["F"]
    fid = {f: i for i, f in enumerate(F)}
    VE = [[] for _ in range(nv)]
    for i, (u, w) in enumerate(E):
        VE[u].append(i)
        VE[w].append(i)
    VF = [[] for _ in range(nv)]
    EF = [[] for _ in range(len(E))]
    eid = {e: i for i, e in enumerate(E)}
    for i, (a, b, c) in enumerate(F):
        for v in (a, b, c):
            VF[v].append(i)
        for e in ((a, b), (a, c), (b, c)):
            EF[eid[e]].append(i)
    FT = [[] for _ in range(len(F))]
    for t in range(rows.shape[0]):
        r = [int(x) for x in rows[t]]
        for i in range(4):
            for j in range(i + 1, 4):
                for k in range(j + 1, 4):
                    FT[fid[(r[i], r[j], r[k])]].append(t)
    return {"VE": [sorted(x) for x in VE], "VF": [sorted(x) for x in VF], "EF": [sorted(x) for x in EF],
            "FT": [sorted(x) for x in FT]}


# ---------------------------------------------------------------------------
# Discrete gradient (Section 5.1, the DiscreteGradient workload: a Forman
# discrete vector field of a vertex scalar field, built lower star by lower
# star).  Reading: the lower star of v is every simplex that contains v and
# whose other vertices all lie below v, "below" meaning a smaller field value
# with ties broken by the smaller input id.  Each lower star is processed on
# its own by the lower-star construction of Robins, Wood and Sheppard (2011,
# "ProcessLowerStars"):
#   * an empty lower star makes v critical;
#   * otherwise v is paired with the lower-star edge of smallest value
#     sequence; every other edge waits in the "zero" queue;
#   * a simplex whose faces inside the lower star are all classified but one
#     enters the "one" queue; popping it pairs it with that face (or, if none
#     is left, moves it to the zero queue);
#   * when the one queue is empty the smallest entry of the zero queue that
#     is still unclassified becomes critical.
# The value sequence of a simplex of the lower star of v is the list of its
# other vertices' (value, input id) keys in decreasing order; sequences
# compare lexicographically, a proper prefix first.  "Faces inside the lower
# star" are the faces that contain v, not counting v itself.
# Plain Python on vertex tuples; meant for small meshes.
# ---------------------------------------------------------------------------

def lower_star_gradient(canon: dict, field, inid, vertices=None) -> dict:
    """{"pairs": [(face, coface), ...], "critical": [simplex, ...]}, every
    simplex a tuple of canonical vertex ids in increasing order.
    field, inid: per canonical vertex.  vertices: the lower stars to process
    (default all; lower stars are disjoint, so any subset is exact)."""
    import heapq
    from itertools import combinations

    rows = canon["rows"]
    nv = int(canon["nv"])
    f = [float(x) for x in np.asarray(field, dtype=np.float64)]
    ids = [int(x) for x in np.asarray(inid)]

    def key(x):
        return (f[x], ids[x])

    todo = range(nv) if vertices is None else [int(v) for v in vertices]
    want = None if vertices is None else set(todo)
    star = {v: [] for v in todo}
    for t in range(rows.shape[0]):
        for x in rows[t]:
            if want is None or int(x) in want:
                star[int(x)].append(t)

    pairs, critical = [], []
    for v in todo:
        kv = key(v)
        low = set()
        for t in star[v]:
            lower = [int(x) for x in rows[t] if int(x) != v and key(int(x)) < kv]
            for r in range(1, len(lower) + 1):
                for c in combinations(lower, r):
                    low.add(tuple(sorted((v,) + c)))
        if not low:
            critical.append((v,))
            continue

        def seq(s):
            return tuple(sorted((key(x) for x in s if x != v), reverse=True))

        # faces of s inside the lower star: drop one vertex other than v
        inner = {s: [tuple(x for x in s if x != w) for w in s if w != v] for s in low}
        inner = {s: [g for g in fs if len(g) > 1] for s, fs in inner.items()}
        cof = {s: [] for s in low}
        for s, fs in inner.items():
            for g in fs:
                cof[g].append(s)
        done = set()

        def open_faces(s):
            return [g for g in inner[s] if g not in done]

        zero, one, in_one = [], [], set()

        def offer_cofaces(s):
            for c in cof[s]:
                if c not in done and c not in in_one and len(open_faces(c)) == 1:
                    heapq.heappush(one, (seq(c), c))
                    in_one.add(c)

        edges = [s for s in low if len(s) == 2]
        first = min(edges, key=seq)
        pairs.append(((v,), first))
        done.add(first)
        for e in edges:
            if e != first:
                heapq.heappush(zero, (seq(e), e))
        offer_cofaces(first)
        while one or zero:
            while one:
                _, a = heapq.heappop(one)
                in_one.discard(a)
                if a in done:
                    continue
                left = open_faces(a)
                if not left:
                    heapq.heappush(zero, (seq(a), a))
                    continue
                g = left[0]
                pairs.append((g, a))
                done.add(g)
                done.add(a)
                offer_cofaces(a)
                offer_cofaces(g)
            while zero:
                _, g = heapq.heappop(zero)
                if g in done:
                    continue
                critical.append(g)
                done.add(g)
                offer_cofaces(g)
                break
    return {"pairs": pairs, "critical": critical}
