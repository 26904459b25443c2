"""GB300 cluster-relation producer (GALE, arXiv 2507.15230) - Python binding.

A thin ctypes layer over the C ABI declared in ``include/gale.h``: argument
marshalling only.  Every step of the producer runs in ``libgale.so`` (host
runtime in C++, kernels in CUDA for sm_103a).  PyTorch supplies the CUDA
stream and, through its caching allocator, the device memory.

There is no fallback: if the library cannot be built or loaded, importing
this module raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

VT, VV, ET, TT = 1, 2, 4, 8
ENUM_SORTED, ENUM_FIRST_APPEARANCE = 0, 1
CB_VE, CB_VF, CB_EF, CB_FT = 1, 2, 4, 8
REL_FE, REL_TE, REL_TF = 1, 2, 3
ALL = 15
MODE_PER_CLUSTER, MODE_BATCHED = 0, 1
SERVE_LOOP, SERVE_BATCH, SERVE_SINGLE = 0, 1, 2
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "EBUSY", 4: "ETIMEOUT", 5: "ENOTFOUND", 6: "ECUDA", 7: "EDEVICE"}
ARRAYS = ("vt_off", "vt_val", "vv_off", "vv_val", "et_uoff", "et_w", "et_off", "et_val", "tt_off", "tt_val")
ARRAY_REL = (VT, VT, VV, VV, ET, ET, ET, ET, TT, TT)

_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class GaleError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Coboundary(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64 * 4), ("len", ctypes.c_int64 * 4), ("off", ctypes.c_void_p * 4),
                ("val", ctypes.c_void_p * 4)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("nt", ctypes.c_int64), ("xyz", ctypes.c_void_p), ("tv", ctypes.c_void_p),
                ("seg", ctypes.c_void_p), ("nclusters", ctypes.c_int32), ("precondition_mask", ctypes.c_uint32),
                ("cache_budget_bytes", ctypes.c_int64), ("stream", ctypes.c_void_p), ("alloc", _ALLOC),
                ("free", _FREE), ("alloc_ctx", ctypes.c_void_p), ("device", ctypes.c_int32),
                ("host_threads", ctypes.c_int32), ("part_vertices", ctypes.c_int32), ("cut_bytes", ctypes.c_int32)]


class View(ctypes.Structure):
    _fields_ = [("cluster", ctypes.c_int32), ("mask", ctypes.c_uint32), ("v_begin", ctypes.c_int32),
                ("v_end", ctypes.c_int32), ("t_begin", ctypes.c_int32), ("t_end", ctypes.c_int32),
                ("n_edges", ctypes.c_int32), ("reserved", ctypes.c_int32)] + \
               [(a, ctypes.c_void_p) for a in ARRAYS] + [("handle", ctypes.c_uint64)]


class Arrays(ctypes.Structure):
    _fields_ = [(a, ctypes.c_void_p) for a in ARRAYS]


class Info(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("nt", ctypes.c_int64), ("nclusters", ctypes.c_int32),
                ("device", ctypes.c_int32), ("n_edges", ctypes.c_int64), ("total", ctypes.c_int64 * 5),
                ("block_bytes", ctypes.c_int64), ("ext_tets", ctypes.c_int64), ("halo_tets", ctypes.c_int64),
                ("nbins", ctypes.c_int32), ("max_cluster_tets", ctypes.c_int32),
                ("load_host_seconds", ctypes.c_double), ("load_device_seconds", ctypes.c_double),
                ("nparts", ctypes.c_int32), ("cut_clusters", ctypes.c_int32)]


class ServeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("requests", "hits", "misses", "builds", "evictions", "batches",
                                              "cache_bytes_used", "cache_bytes_budget", "max_batch", "prefetches",
                                              "prefetch_hits", "prefetch_dropped", "leases_expired",
                                              "t_enqueue_ns", "t_queue_ns", "t_prepare_ns", "t_build_ns", "t_kernel_ns",
                                              "t_wait_ns", "max_wait_ns")] + [("depth_hist", ctypes.c_int64 * 12)] + \
               [("max_queue_ns", ctypes.c_int64), ("queue_hist", ctypes.c_int64 * 16)] + \
               [(n, ctypes.c_int64) for n in ("leader_passes", "leader_hold_ns", "max_leader_hold_ns", "promotions",
                                              "max_prefetch_queue", "requester_pumps")]


# the symbols include/gale.h declares
EXPORTS = ("gale_load_mesh", "gale_build_clusters", "gale_build_clusters_noalloc", "gale_synchronize", "gale_bulk_view", "gale_bulk_arrays",
           "gale_bulk_export", "gale_copy_to_host", "gale_build_export", "gale_request", "gale_release", "gale_serve_stats_get", "gale_get_permutations",
           "gale_get_intervals", "gale_get_rows", "gale_get_working_set", "gale_get_info", "gale_set_tuning",
           "gale_autotune", "gale_get_bins", "gale_get_bin_members", "gale_set_teams", "gale_enumerate", "gale_get_enumeration",
           "gale_boundary", "gale_build_coboundary", "gale_serve_configure", "gale_serve_set_lease", "gale_stream", "gale_last_launch_count", "gale_destroy", "gale_last_error")

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build: bool = True):
    """Load (building first if needed) libgale.so; raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libgale.so not found at {path}")
    lib = ctypes.CDLL(path)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    lib.gale_load_mesh.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(P)]
    lib.gale_build_clusters.argtypes = [P, P, i32, u32, i32]
    lib.gale_synchronize.argtypes = [P]
    lib.gale_build_clusters_noalloc.argtypes = [P, P, i32, u32, ctypes.POINTER(Arrays), P]
    lib.gale_bulk_view.argtypes = [P, i32, ctypes.POINTER(View)]
    lib.gale_bulk_arrays.argtypes = [P, ctypes.POINTER(Arrays), P]
    lib.gale_bulk_export.argtypes = [P, u32, ctypes.POINTER(Arrays)]
    lib.gale_copy_to_host.argtypes = [P, P, P, ctypes.c_size_t]
    lib.gale_build_export.argtypes = [P, P, ctypes.c_int32, u32, ctypes.POINTER(Arrays), ctypes.c_int32]
    lib.gale_request.argtypes = [P, i32, u32, i64, ctypes.POINTER(View)]
    lib.gale_release.argtypes = [P, ctypes.POINTER(View)]
    lib.gale_serve_stats_get.argtypes = [P, ctypes.POINTER(ServeStats)]
    lib.gale_get_permutations.argtypes = [P, P, P]
    lib.gale_get_intervals.argtypes = [P, P, P, P]
    lib.gale_get_rows.argtypes = [P, P]
    lib.gale_get_working_set.argtypes = [P, i32, P, ctypes.POINTER(i64), P, ctypes.POINTER(i64)]
    lib.gale_get_info.argtypes = [P, ctypes.POINTER(Info)]
    lib.gale_set_tuning.argtypes = [P, i32, i32]
    lib.gale_set_teams.argtypes = [P, i32, i32]
    lib.gale_autotune.argtypes = [P, u32, i32, P, i32]
    lib.gale_get_bin_members.argtypes = [P, P]
    lib.gale_enumerate.argtypes = [P, i32]
    lib.gale_get_enumeration.argtypes = [P, P, P, P, P, P]
    lib.gale_boundary.argtypes = [P, i32, P, i64, P]
    lib.gale_build_coboundary.argtypes = [P, u32, ctypes.POINTER(Coboundary)]
    lib.gale_get_bins.argtypes = [P, P, i32, ctypes.POINTER(i32)]
    lib.gale_serve_configure.argtypes = [P, i32, i64, i32, i32]
    lib.gale_serve_set_lease.argtypes = [P, i64]
    lib.gale_stream.argtypes = [P]
    lib.gale_stream.restype = P
    lib.gale_last_launch_count.argtypes = [P]
    lib.gale_last_launch_count.restype = i64
    lib.gale_destroy.argtypes = [P]
    lib.gale_destroy.restype = None
    lib.gale_last_error.argtypes = []
    lib.gale_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("gale_stream", "gale_last_launch_count", "gale_destroy", "gale_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise GaleError(rc, _lib.gale_last_error().decode(errors="replace"))


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


class _DevArray:
    """A device int32 range exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<i4", "data": (int(ptr) if n else 0, False),
                                         "version": 3}


def device_tensor(ptr: int, n: int):
    """torch int32 tensor aliasing n elements of device memory at ptr."""
    import torch
    if n == 0:
        return torch.zeros(0, dtype=torch.int32, device="cuda")
    return torch.as_tensor(_DevArray(ptr, n), device="cuda")


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, handed to the C ABI."""

    def __init__(self, device: int, stream: int):
        import torch
        self.device, self.stream = device, stream
        self._torch = torch

        def alloc(_ctx, nbytes):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), device, stream))
            except Exception:
                return None

        def free(_ctx, ptr):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = _ALLOC(alloc)
        self.free = _FREE(free)


@dataclass
class Mesh:
    """Input arrays in the paper's form (Section 4.3): V, T (TV), S."""
    xyz: np.ndarray | None
    tv: np.ndarray
    seg: np.ndarray
    nclusters: int


class Context:
    """A loaded mesh (one gale_ctx).  Use ``Context.load``."""

    def __init__(self, handle, lib, keep):
        self._h = handle
        self._lib = lib
        self._keep = keep  # arrays and callbacks that must outlive the handle
        self.nv = self.info().nv
        self.nt = self.info().nt
        self.K = self.info().nclusters

    # ---------------- construction ----------------
    @classmethod
    def load(cls, mesh, precondition_mask: int = ALL, device: int = 0, stream=None, cache_budget_bytes: int = 0,
             host_threads: int = 0, torch_alloc: bool = True, part_vertices: int = 0,
             cut_bytes: int = 0) -> "Context":
        """gale_load_mesh.  mesh: anything with tv, seg, nclusters (and
        optionally xyz).  device=-1 makes a host-only context.  stream: a
        torch.cuda.Stream or raw handle; defaults to torch's current stream.
        part_vertices / cut_bytes: how clusters too large for one CTA are cut
        into parts for batched builds (0 = defaults, part_vertices < 0 =
        never)."""
        lib = load_library()
        tv = np.ascontiguousarray(mesh.tv, dtype=np.int32).reshape(-1, 4)
        seg = np.ascontiguousarray(mesh.seg, dtype=np.int32)
        xyz = None if getattr(mesh, "xyz", None) is None else np.ascontiguousarray(mesh.xyz, dtype=np.float32)
        d = MeshDesc()
        d.nv, d.nt = seg.shape[0], tv.shape[0]
        d.xyz = _p(xyz) if xyz is not None else None
        d.tv = _p(tv) if tv.size else None
        d.seg = _p(seg)
        d.nclusters = int(mesh.nclusters)
        d.precondition_mask = precondition_mask
        d.cache_budget_bytes = cache_budget_bytes
        d.device = device
        d.host_threads = host_threads
        d.part_vertices = part_vertices
        d.cut_bytes = cut_bytes
        keep = [tv, seg, xyz]
        if device >= 0:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("CUDA device requested but torch sees no GPU")
            torch.cuda.set_device(device)
            if stream is None:
                stream = torch.cuda.current_stream(device)
            sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
            d.stream = sh
            if torch_alloc:
                ta = _TorchAllocator(device, sh)
                d.alloc, d.free = ta.alloc, ta.free
                keep.append(ta)
        h = ctypes.c_void_p()
        _check(lib.gale_load_mesh(ctypes.byref(d), ctypes.byref(h)))
        return cls(h, lib, keep)

    def close(self):
        if self._h:
            self._lib.gale_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------- builds ----------------
    def build(self, ids=None, mask: int = ALL, mode: int = MODE_BATCHED):
        """gale_build_clusters (asynchronous on the context stream)."""
        if ids is None:
            _check(self._lib.gale_build_clusters(self._h, None, 0, mask, mode))
        else:
            ids = np.ascontiguousarray(ids, dtype=np.int32)
            _check(self._lib.gale_build_clusters(self._h, _p(ids), ids.shape[0], mask, mode))

    def build_noalloc(self, ids, mask: int, out: dict):
        """gale_build_clusters_noalloc: build into caller-owned device arrays
        (out: array name -> CUDA int32 tensor or None) without any allocation;
        each tensor's element count is passed as that array's capacity."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        a = Arrays()
        lengths = np.zeros(len(ARRAYS), dtype=np.int64)
        for n, t in out.items():
            if t is None:
                continue
            setattr(a, n, t.data_ptr() if t.numel() else None)
            lengths[ARRAYS.index(n)] = t.numel()
        _check(self._lib.gale_build_clusters_noalloc(self._h, _p(ids), ids.shape[0], mask, ctypes.byref(a),
                                                     _p(lengths)))

    def synchronize(self):
        _check(self._lib.gale_synchronize(self._h))

    @property
    def stream_handle(self) -> int:
        return self._lib.gale_stream(self._h) or 0

    def last_launch_count(self) -> int:
        return int(self._lib.gale_last_launch_count(self._h))

    def bulk_view(self, index: int) -> View:
        v = View()
        _check(self._lib.gale_bulk_view(self._h, index, ctypes.byref(v)))
        return v

    def bulk_arrays(self):
        """(dict name -> device pointer, dict name -> length) of the last bulk build."""
        a = Arrays()
        L = np.zeros(10, np.int64)
        _check(self._lib.gale_bulk_arrays(self._h, ctypes.byref(a), _p(L)))
        return {n: getattr(a, n) or 0 for n in ARRAYS}, {n: int(L[i]) for i, n in enumerate(ARRAYS)}

    def export(self, mask: int = ALL, out: dict | None = None) -> dict:
        """gale_bulk_export into host numpy arrays (allocated unless given)."""
        _, L = self.bulk_arrays()
        if out is None:
            out = {n: np.empty(L[n], np.int32) for i, n in enumerate(ARRAYS) if mask & ARRAY_REL[i]}
        a = Arrays()
        for n, arr in out.items():
            setattr(a, n, _p(arr) if arr.size else None)
        _check(self._lib.gale_bulk_export(self._h, mask, ctypes.byref(a)))
        return out

    def build_export(self, ids=None, mask: int = ALL, out: dict | None = None, chunks: int = 0) -> dict:
        """gale_build_export: build the listed clusters (None: all) and copy
        the outputs into host numpy arrays, chunk copies overlapping the
        build (allocated unless given; pinned buffers give the overlap)."""
        if ids is None:
            idp, n = None, 0
        else:
            ids = np.ascontiguousarray(ids, dtype=np.int32)
            idp, n = _p(ids), int(ids.size)
        if out is None:
            lens = self.output_lengths(ids, mask)
            out = {nm: np.empty(lens[nm], np.int32) for i, nm in enumerate(ARRAYS) if mask & ARRAY_REL[i]}
        a = Arrays()
        for nm, arr in out.items():
            setattr(a, nm, _p(arr) if arr.size else None)
        _check(self._lib.gale_build_export(self._h, idp, n, mask, ctypes.byref(a), chunks))
        return out

    def output_lengths(self, ids=None, mask: int = ALL) -> dict:
        """Element counts of the ten bulk arrays a build of ids would fill."""
        I_V, I_T, sizes = self.intervals()
        ks = np.arange(self.K) if ids is None else np.asarray(ids, dtype=np.int64)
        nvo = (I_V[ks + 1] - I_V[ks]).astype(np.int64)
        nown = (I_T[ks + 1] - I_T[ks]).astype(np.int64)
        sz = sizes[ks]
        n_e = sz[:, 2]
        per = [nvo + 1, sz[:, 0], nvo + 1, sz[:, 1], nvo + 1, n_e, n_e + 1, sz[:, 3], nown + 1, sz[:, 4]]
        L = {nm: int(per[i].sum()) if mask & ARRAY_REL[i] else 0 for i, nm in enumerate(ARRAYS)}
        return L

    def bulk_offsets(self, index: int) -> dict:
        """Element offsets of the index-th cluster in each bulk array."""
        ptrs, _ = self.bulk_arrays()
        v = self.bulk_view(index)
        res = {}
        for n in ARRAYS:
            p = getattr(v, n)
            res[n] = None if not p else (p - ptrs[n]) // 4
        return res

    # ---------------- serving ----------------
    def request(self, cluster: int, mask: int, timeout_ns: int = 0) -> View:
        v = View()
        _check(self._lib.gale_request(self._h, cluster, mask, timeout_ns, ctypes.byref(v)))
        return v

    def serve_configure(self, mode: int, idle_us: int = 0, loop_ctas: int = 0, prefetch: int = 0):
        """gale_serve_configure (before the first request)."""
        _check(self._lib.gale_serve_configure(self._h, mode, idle_us, loop_ctas, prefetch))

    def serve_set_lease(self, lease_ns: int):
        """gale_serve_set_lease: pins of later requests expire after lease_ns (0: never)."""
        _check(self._lib.gale_serve_set_lease(self._h, int(lease_ns)))

    def release(self, view: View):
        _check(self._lib.gale_release(self._h, ctypes.byref(view)))

    def serve_stats(self) -> ServeStats:
        s = ServeStats()
        _check(self._lib.gale_serve_stats_get(self._h, ctypes.byref(s)))
        return s

    # ---------------- introspection ----------------
    def info(self) -> Info:
        i = Info()
        _check(self._lib.gale_get_info(self._h, ctypes.byref(i)))
        return i

    def permutations(self):
        vp = np.empty(self.nv, np.int32)
        tp = np.empty(max(self.nt, 1), np.int32)
        _check(self._lib.gale_get_permutations(self._h, _p(vp), _p(tp)))
        return vp, tp[:self.nt]

    def intervals(self):
        I_V = np.empty(self.K + 1, np.int64)
        I_T = np.empty(self.K + 1, np.int64)
        sizes = np.empty((self.K, 5), np.int64)
        _check(self._lib.gale_get_intervals(self._h, _p(I_V), _p(I_T), _p(sizes)))
        return I_V, I_T, sizes

    def rows(self) -> np.ndarray:
        r = np.empty((max(self.nt, 1), 4), np.int32)
        _check(self._lib.gale_get_rows(self._h, _p(r)))
        return r[:self.nt]

    def working_set(self, k: int):
        ne, nh = ctypes.c_int64(0), ctypes.c_int64(0)
        rc = self._lib.gale_get_working_set(self._h, k, None, ctypes.byref(ne), None, ctypes.byref(nh))
        ext = np.empty(max(ne.value, 1), np.int32)
        halo = np.empty(max(nh.value, 1), np.int32)
        _check(self._lib.gale_get_working_set(self._h, k, _p(ext), ctypes.byref(ne), _p(halo), ctypes.byref(nh)))
        return ext[:ne.value], halo[:nh.value]

    def bins(self) -> list:
        """Size bins: members, threads, working bytes per CTA, CTAs per SM,
        grid, spill (1: working memory in global scratch), per_item (1: each
        member runs under its own plan), parts (members that are parts of cut
        clusters; -1: a bin of the cut clusters themselves, which batched
        builds skip), teams (clusters per CTA of its batched launches; 0:
        one)."""
        n = ctypes.c_int32(0)
        _check(self._lib.gale_get_bins(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros(9 * max(n.value, 1), np.int32)
        _check(self._lib.gale_get_bins(self._h, _p(out), n.value, ctypes.byref(n)))
        keys = ("clusters", "threads", "bytes", "ctas_per_sm", "grid", "spill", "per_item", "parts", "teams")
        return [dict(zip(keys, out[9 * i:9 * i + 9].tolist())) for i in range(n.value)]

    def set_teams(self, team_threads: int, teams: int):
        """gale_set_teams: several small clusters per CTA in batched builds
        (teams of team_threads threads; teams = 0 turns it off)."""
        _check(self._lib.gale_set_teams(self._h, team_threads, teams))

    def bin_members(self) -> np.ndarray:
        """Work item ids of bin 0, bin 1, ... in launch order: clusters
        (ids below K), then parts of cut clusters (id K + p)."""
        n = self.K + int(self.info().nparts)
        out = np.empty(max(n, 1), np.int32)
        _check(self._lib.gale_get_bin_members(self._h, _p(out)))
        return out[:n]

    def enumerate(self, order: int = 0) -> dict:
        """gale_enumerate + gale_get_enumeration: E (nE x 2), F (nF x 3),
        I_E, I_F (K+1) in canonical ids; order ENUM_SORTED or
        ENUM_FIRST_APPEARANCE."""
        _check(self._lib.gale_enumerate(self._h, order))
        return self.enumeration()

    def enumeration(self) -> dict:
        """gale_get_enumeration of the last gale_enumerate (ENOTFOUND before)."""
        counts = np.zeros(2, np.int64)
        _check(self._lib.gale_get_enumeration(self._h, _p(counts), None, None, None, None))
        E = np.empty((max(int(counts[0]), 1), 2), np.int32)
        F = np.empty((max(int(counts[1]), 1), 3), np.int32)
        I_E = np.empty(self.K + 1, np.int64)
        I_F = np.empty(self.K + 1, np.int64)
        _check(self._lib.gale_get_enumeration(self._h, None, _p(E), _p(I_E), _p(F), _p(I_F)))
        return {"E": E[:counts[0]], "F": F[:counts[1]], "I_E": I_E, "I_F": I_F}

    def boundary(self, relation: int, ids) -> np.ndarray:
        """gale_boundary: REL_FE (3 per triangle), REL_TE (6 per tet) or
        REL_TF (4 per tet)."""
        width = {REL_FE: 3, REL_TE: 6, REL_TF: 4}[relation]
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        out = np.empty((max(ids.size, 1), width), np.int32)
        _check(self._lib.gale_boundary(self._h, relation, _p(ids) if ids.size else None, ids.size, _p(out)))
        return out[:ids.size]

    def copy_to_host(self, dev_ptr: int, n: int, out: np.ndarray | None = None) -> np.ndarray:
        """gale_copy_to_host of n int32 elements at a device pointer the
        library handed out, into `out` (a new array unless given)."""
        if out is None:
            out = np.empty(n, np.int32)
        assert out.dtype == np.int32 and out.size >= n and out.flags["C_CONTIGUOUS"]
        if n:
            _check(self._lib.gale_copy_to_host(self._h, _p(out), dev_ptr, 4 * n))
        return out[:n]

    def coboundary(self, which: int = CB_VE | CB_VF | CB_EF | CB_FT) -> dict:
        """gale_build_coboundary: {"VE"|"VF"|"EF"|"FT": (offsets, values)} as
        host numpy arrays (copied with gale_copy_to_host)."""
        c = Coboundary()
        _check(self._lib.gale_build_coboundary(self._h, which, ctypes.byref(c)))
        out = {}
        for i, name in enumerate(("VE", "VF", "EF", "FT")):
            if which & (1 << i):
                n, ln = int(c.rows[i]), int(c.len[i])
                out[name] = (self.copy_to_host(c.off[i], n + 1), self.copy_to_host(c.val[i], ln))
        return out

    def set_tuning(self, threads: int = 0, ctas_per_sm: int = 0):
        _check(self._lib.gale_set_tuning(self._h, threads, ctas_per_sm))

    def autotune(self, mask: int = ALL, reps: int = 2) -> list:
        """gale_autotune: per size bin, the fastest block size and CTAs per
        SM; returns the chosen build time (ms) of each bin."""
        nb = len(self.bins())
        best = np.zeros(max(nb, 1), np.float32)
        _check(self._lib.gale_autotune(self._h, mask, reps, _p(best), nb))
        return [float(x) for x in best[:nb]]


def view_to_numpy(view: View) -> dict:
    """Copy one view's device arrays to host numpy (through torch)."""
    nvo = view.v_end - view.v_begin
    nown = view.t_end - view.t_begin
    out = {}

    def grab(name, n):
        p = getattr(view, name)
        if not p:
            return None
        return device_tensor(p, n).cpu().numpy()

    if view.mask & VT:
        out["vt_off"] = grab("vt_off", nvo + 1)
        out["vt_val"] = grab("vt_val", int(out["vt_off"][-1]))
    if view.mask & VV:
        out["vv_off"] = grab("vv_off", nvo + 1)
        out["vv_val"] = grab("vv_val", int(out["vv_off"][-1]))
    if view.mask & ET:
        out["et_uoff"] = grab("et_uoff", nvo + 1)
        ne = view.n_edges
        out["et_w"] = grab("et_w", ne)
        out["et_off"] = grab("et_off", ne + 1)
        out["et_val"] = grab("et_val", int(out["et_off"][-1]))
    if view.mask & TT:
        out["tt_off"] = grab("tt_off", nown + 1)
        out["tt_val"] = grab("tt_val", int(out["tt_off"][-1]))
    return out
