/*
 * gale.h - C ABI of the GB300 cluster-relation producer.
 *
 * The library is the producer side of a GPU-aided localized data structure
 * for tetrahedral meshes (GALE, Section 4).  Consumers ask for the
 * coboundary / adjacency relations of whole mesh segments ("clusters", the
 * paper's segments of Section 4.3); the library builds them on the GPU as
 * canonical, index-sorted CSR:
 *
 *   VT(v)    tets incident to vertex v             (coboundary, Table 1)
 *   VV(v)    vertices adjacent to v                (adjacency,  Table 1)
 *   ET(u,w)  tets incident to edge (u,w), u < w    (coboundary, Table 1)
 *   TT(t)    tets sharing a triangle with tet t    (adjacency,  Table 1)
 *
 * Conventions for every call:
 *  - All ids in outputs are CANONICAL ids (see gale_load_mesh).  The
 *    permutations back to input ids come from gale_get_permutations; applying
 *    them is the paper's local-to-global mapping step (Section 4.5).
 *  - Every row is ascending.  Offset arrays are int32, relative to their
 *    cluster (the first offset of every cluster is 0).
 *  - No call throws; every failure returns a status and sets a thread-local
 *    message readable with gale_last_error().
 *  - Host pointers are caller-owned and are only read during the call.
 *    Device pointers returned by the library stay library-owned.
 */
#ifndef GALE_H
#define GALE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GALE_OK = 0,
    GALE_EINVAL = 1,    /* invalid argument or invalid mesh */
    GALE_ENOMEM = 2,    /* device or host allocation failed, or over budget */
    GALE_EBUSY = 3,     /* cache budget fully pinned; retry after releases */
    GALE_ETIMEOUT = 4,  /* a wait ran past its deadline */
    GALE_ENOTFOUND = 5, /* no such cluster / view / symbol */
    GALE_ECUDA = 6,     /* a CUDA runtime call failed */
    GALE_EDEVICE = 7    /* a kernel reported an error word (see message) */
} gale_status;

/* Relation mask bits. */
enum { GALE_VT = 1u, GALE_VV = 2u, GALE_ET = 4u, GALE_TT = 8u, GALE_ALL = 15u };

/* Build forms of gale_build_clusters. */
enum {
    GALE_MODE_PER_CLUSTER = 0, /* one kernel launch per cluster (baseline form) */
    GALE_MODE_BATCHED = 1      /* persistent size-binned kernels, replayed from a captured CUDA graph */
};

/* Device allocator hooks: return device memory aligned to 256 bytes, or NULL. */
typedef void *(*gale_alloc_fn)(void *alloc_ctx, size_t bytes);
typedef void (*gale_free_fn)(void *alloc_ctx, void *ptr);

typedef struct gale_ctx gale_ctx; /* opaque; one per loaded mesh */

/*
 * Mesh description (Section 4.3, "Input data"): V, T (the TV relation) and
 * S.  All arrays are HOST memory, caller-owned, read only during
 * gale_load_mesh.
 *   nv, nt            vertex and tet counts (1 <= nv, 0 <= nt, both < 2^31)
 *   xyz               float[nv*3] coordinates; may be NULL (not used by the
 *                     producer, kept for consumers)
 *   tv                int32[nt*4] vertex ids of each tet, any order
 *   seg               int32[nv] segment (cluster) id of each vertex, in
 *                     [0, nclusters)
 *   precondition_mask relations the context will serve (Section 4.3,
 *                     preconditioning); only their working data is built
 *   cache_budget_bytes HBM budget of the serving relation cache
 *                     (gale_request); 0 disables serving
 *   stream            cudaStream_t every kernel and copy of this context is
 *                     ordered on; NULL = a stream the library creates
 *   alloc/free        device allocator hooks; NULL = cudaMalloc / cudaFree
 *   device            CUDA device ordinal; -1 makes a HOST-ONLY context that
 *                     runs the host-side initialisation and nothing else
 *   host_threads      threads for host-side initialisation, 0 = all cores
 *   part_vertices     a cluster whose working set would not fit one CTA's
 *                     shared memory (estimated shared memory above cut_bytes)
 *                     is also cut into parts of about this many own vertices
 *                     (contiguous canonical ranges); batched builds build the
 *                     parts, each on its own CTA, straight into the cluster's
 *                     outputs.  0 = 256; negative = never cut
 *   cut_bytes         0 = 160 KB
 */
typedef struct {
    int64_t nv, nt;
    const float *xyz;
    const int32_t *tv;
    const int32_t *seg;
    int32_t nclusters;
    uint32_t precondition_mask;
    int64_t cache_budget_bytes;
    void *stream;
    gale_alloc_fn alloc;
    gale_free_fn free;
    void *alloc_ctx;
    int32_t device;
    int32_t host_threads;
    int32_t part_vertices;
    int32_t cut_bytes;
} gale_mesh_desc;

/*
 * One cluster's relations.  Device pointers, valid until gale_release (views
 * from gale_request) or until the next gale_build_clusters / gale_destroy
 * (views from gale_bulk_view).  Pointers for relations not in `mask` are NULL.
 *   vt_off[nv_own+1], vt_val      VT rows of vertices v_begin .. v_end-1
 *   vv_off[nv_own+1], vv_val      VV rows of the same vertices
 *   et_uoff[nv_own+1]             edges of each vertex u as lower endpoint
 *   et_w[n_edges]                 upper endpoint w of each edge (u, w)
 *   et_off[n_edges+1], et_val     ET rows of those edges
 *   tt_off[t_end-t_begin+1], tt_val  TT rows of the cluster's internal tets
 */
typedef struct {
    int32_t cluster;
    uint32_t mask;
    int32_t v_begin, v_end; /* canonical vertex ids of the cluster (I_V interval) */
    int32_t t_begin, t_end; /* canonical ids of its internal tets (I_T interval) */
    int32_t n_edges;        /* edges whose lower endpoint it owns (I_E difference) */
    int32_t reserved;
    const int32_t *vt_off, *vt_val, *vv_off, *vv_val;
    const int32_t *et_uoff, *et_w, *et_off, *et_val;
    const int32_t *tt_off, *tt_val;
    uint64_t handle; /* non-zero for views that pin a cache entry */
} gale_view;

/* The ten output arrays of a bulk build (device or host pointers). */
typedef struct {
    int32_t *vt_off, *vt_val, *vv_off, *vv_val;
    int32_t *et_uoff, *et_w, *et_off, *et_val;
    int32_t *tt_off, *tt_val;
} gale_arrays;

/* Counts and sizes of a context. */
typedef struct {
    int64_t nv, nt;
    int32_t nclusters;
    int32_t device;
    int64_t n_edges;           /* edges of the whole mesh */
    int64_t total[5];          /* entries of VT, VV, edges, ET, TT over all clusters */
    int64_t block_bytes;       /* device bytes of the cluster working sets */
    int64_t ext_tets, halo_tets; /* sum of |T_ex(k)| and of |halo(k)| */
    int32_t nbins;             /* size bins of the batched form */
    int32_t max_cluster_tets;  /* largest working set (tets) */
    double load_host_seconds;  /* host-side initialisation time */
    double load_device_seconds;/* upload + size pass time */
    int32_t nparts;            /* parts of the clusters cut for batched builds */
    int32_t cut_clusters;      /* clusters cut into parts */
} gale_info;

/* Per-call statistics of the serving path. */
typedef struct {
    int64_t requests, hits, misses, builds, evictions, batches;
    int64_t cache_bytes_used, cache_bytes_budget;
    int64_t max_batch;
    int64_t prefetches;        /* entries built ahead of any request (proactive prefetch) */
    int64_t prefetch_hits;     /* requests served by such an entry, ready or in flight */
    int64_t prefetch_dropped;  /* prefetches dropped because the budget was full (a prefetch never evicts) */
    int64_t leases_expired;    /* pins revoked because their lease ran out (gale_serve_set_lease) */
    /* Waiting time by stage (the stages of Section 5.3's breakdown), in
     * nanoseconds summed over requests or over entries built for a request: */
    int64_t t_enqueue_ns;      /* per request: taking the serving lock, finding or queueing its entry */
    int64_t t_queue_ns;        /* per built entry: queued until admitted (budget, ring space, leader) */
    int64_t t_prepare_ns;      /* per built entry: admission, slot placement, publication or launch */
    int64_t t_build_ns;        /* per built entry: on the device until the leader saw it done */
    int64_t t_kernel_ns;       /* per entry built by the device loop: its build alone, from the
                                  CTA's claim to its completion (device clock) */
    int64_t t_wait_ns;         /* per request: from the call to its return */
    int64_t max_wait_ns;       /* the longest single request */
    /* Queue length (the paper's queue statistics, Section 4.5): each leader
     * pass with work pending counts once in bucket b of the number of
     * entries queued or in flight, b = 0 for 1, 1 for 2-3, 2 for 4-7, ...,
     * 11 for 2048 and more. */
    int64_t depth_hist[12];
    /* The leader's own timing: */
    int64_t max_queue_ns;      /* the longest admission wait of an entry built for a request */
    int64_t queue_hist[16];    /* admission waits of entries built for a request: bucket b counts
                                  waits of [2^b, 2^(b+1)) microseconds (b = 0 also below 1 us) */
    int64_t leader_passes;     /* passes of the leader loop */
    int64_t leader_hold_ns;    /* summed time the leader held the serving lock in its passes */
    int64_t max_leader_hold_ns;/* the longest single pass */
    int64_t promotions;        /* queued prefetches a request moved to the request queue */
    int64_t max_prefetch_queue;/* the longest prefetch queue seen */
    int64_t requester_pumps;   /* steps of the serving state machine run by waiting requests */
} gale_serve_stats;

/*
 * gale_load_mesh - initialisation (Section 4.3, "Initialization").
 * Validates the input (EINVAL on an id out of range, a repeated vertex in a
 * tet, a segment id out of range or two tets with the same vertex set) and
 * builds the canonical numbering:
 *   - vertices ordered by (segment, input id), so segment k owns the
 *     contiguous interval [I_V[k], I_V[k+1]) the interval array I_V of
 *     Section 4.3 presupposes;
 *   - each tet row relabelled and sorted ascending; a tet is internal to the
 *     segment of its lowest vertex (Section 4.3) and tets are ordered by
 *     (owning segment, input index), giving I_T;
 *   - per cluster: its internal tets, its external tets T_ex (Section 4.3),
 *     and the halo of tets outside the cluster that share a triangle with an
 *     internal tet (needed for complete TT rows);
 *   - the exact size of every relation in the precondition mask of every
 *     cluster (a counting pass on the GPU), used for output placement and
 *     cache admission.
 * The cluster working sets are copied to device memory once, as the paper
 * copies its initialised arrays to GPU global memory.  TT of a non-manifold
 * mesh (a triangle in three or more tets) is built as defined: every tet
 * sharing three vertices with t.  A cluster with such a triangle among its
 * internal tets' faces finds its TT rows by a slower pass over its block.
 * Parts of a cut cluster (too large for one CTA) assume at most one
 * partner per face: when the counting pass finds such a triangle in a cut
 * cluster (GALE_TT preconditioned), the load starts again with cutting off
 * (as part_vertices < 0), and the large clusters run whole from global
 * scratch.
 * Size limits, each EINVAL with the cluster named: a cluster's working set
 * (its tets, external tets and halo) holds at most 65534 tets and 65535
 * vertices (16-bit local ids), and no vertex may have more than 255
 * distinct neighbours above it (8-bit edge ranks); use smaller clusters.
 * On success *out owns all of it; release with gale_destroy.
 */
gale_status gale_load_mesh(const gale_mesh_desc *desc, gale_ctx **out);

/*
 * gale_build_clusters - producer kernels (Section 4.6) for a batch of
 * clusters.  ids: HOST int32[n] cluster ids (NULL with n <= 0 = all clusters
 * in order); each id at most once.  mask: relations to build (GALE_* bits,
 * within the precondition mask).  mode: GALE_MODE_PER_CLUSTER or
 * GALE_MODE_BATCHED.  The relations are written to library-owned bulk arrays,
 * clusters consecutively in list order.  The work is ENQUEUED on the
 * context's stream and the call returns; gale_synchronize waits for it and
 * reports kernel errors.  EINVAL on a bad id, mode or mask; ENOMEM if the bulk
 * arrays cannot be allocated.
 */
gale_status gale_build_clusters(gale_ctx *ctx, const int32_t *ids, int32_t n, uint32_t mask, int32_t mode);

/*
 * gale_build_clusters_noalloc - the batched build without any allocation.
 * The paper has no counterpart; this exists for callers that cannot allocate
 * device memory when they need relations: a serving thread that must not
 * synchronise the GPU (cudaMalloc / cudaFree may), an application whose own
 * pool owns all of HBM, or code running where allocation is forbidden.
 *   ids      HOST int32[n], 1 <= n <= 4096 cluster ids (a repeated id is
 *            built into each of its slots); EINVAL beyond 4096.  Only
 *            clusters whose size bin runs in shared memory are accepted:
 *            EINVAL for a cluster of a spill bin (gale_get_bins reports 1 as
 *            a bin's sixth value; gale_get_bin_members lists its clusters)
 *   mask     relations to build (within the precondition mask)
 *   dev_out  caller-owned DEVICE arrays, one per requested relation array,
 *            laid out as the bulk arrays of gale_build_clusters for the same
 *            list: clusters consecutive in list order, offsets relative to
 *            their cluster; the arrays of relations outside mask may be NULL
 *   lengths  HOST int64[10]: how many int32 elements each dev_out array
 *            holds (same order as gale_arrays; entries of relations outside
 *            mask are ignored).  Each requested array must hold at least the
 *            summed lengths that the sizes of gale_get_intervals give for
 *            the list (e.g. vt_off: sum of (v_end - v_begin + 1), vt_val: sum
 *            of the VT sizes); EINVAL otherwise, before anything is copied or
 *            launched
 * The work items, order lists, ticket counters and error word live in one
 * fixed array of about 430 KB of device memory that every GPU which loads
 * the library holds until the process exits; every call reuses it, so calls
 * that overlap on the GPU of one device (from several threads, or from
 * several contexts on that device) race and must be serialised by the
 * caller.  The first call on each device looks up that array's device
 * address; make that first call before any stream capture.  The call returns
 * after the build has finished (it synchronises the context stream); EDEVICE
 * if a kernel reported an error.
 */
gale_status gale_build_clusters_noalloc(gale_ctx *ctx, const int32_t *ids, int32_t n, uint32_t mask,
                                        const gale_arrays *dev_out, const int64_t *lengths);

/* Wait for all work of the context's stream; EDEVICE if a kernel set its
 * error word (the word is cleared), ECUDA on a CUDA error. */
gale_status gale_synchronize(gale_ctx *ctx);

/* View of the index-th cluster of the last bulk build (no pinning). */
gale_status gale_bulk_view(gale_ctx *ctx, int32_t index, gale_view *out);

/* Device pointers and element counts (lengths[10], same order as
 * gale_arrays) of the last bulk build's output arrays. */
gale_status gale_bulk_arrays(gale_ctx *ctx, gale_arrays *dev, int64_t *lengths);

/* Copy the last bulk build's arrays selected by mask into caller HOST
 * buffers (each at least the length gale_bulk_arrays reports; pinned memory
 * is fastest).  Ordered after the build on the context stream; blocks until
 * the copies are done. */
gale_status gale_bulk_export(gale_ctx *ctx, uint32_t mask, const gale_arrays *host_dst);

/* Copy `bytes` from device memory `src` (an array the library handed out:
 * a gale_view, gale_bulk_arrays or gale_coboundary pointer) to caller HOST
 * memory `dst`, ordered after earlier work on the context stream; returns
 * when the copy is complete.  Page-locked destinations take one copy.
 * Pageable ones of 32 MB or more go through two 128 MB pinned staging
 * buffers that the context allocates on first use and keeps until
 * gale_destroy: the copy engine fills one while the host threads move the
 * other into place.  gale_bulk_export copies the same way.  EINVAL for
 * NULL pointers with bytes > 0 or a host-only context; ENOMEM if the
 * staging buffers cannot be allocated; ECUDA if a copy fails. */
gale_status gale_copy_to_host(gale_ctx *ctx, void *dst, const void *src, size_t bytes);

/* Build the listed clusters (ids == NULL or n <= 0: all, in id order) for
 * the relations in mask and copy every output array to caller HOST buffers,
 * overlapping the copy of each finished chunk of clusters with the build of
 * the next one.  This is the paper's kernel-then-copy-back step for a whole
 * batch ("Kernel computation", Section 4.6: the relations are computed on
 * the GPU and returned to the consumers' host memory).
 *   host_dst  one buffer per array of mask, laid out as a bulk build lays
 *             out the device arrays (lengths as gale_bulk_arrays reports after
 *             the call); pinned memory is needed for the overlap.
 *   chunks    0 = automatic (about 256 MB of output per chunk, at most 16),
 *             else 1..64.
 * Afterwards the device bulk arrays hold the same result as after
 * gale_build_clusters(ctx, ids, n, mask, GALE_MODE_BATCHED).  Blocks until
 * the copies are done; EDEVICE if a kernel reported an error. */
gale_status gale_build_export(gale_ctx *ctx, const int32_t *ids, int32_t n, uint32_t mask,
                              const gale_arrays *host_dst, int32_t chunks);

/*
 * gale_request - a consumer's request for the relations of one cluster
 * (Section 4.4: coboundary and adjacency relations are requested for the
 * whole segment).  Thread safe; blocks until the relations are resident or
 * timeout_ns passes (ETIMEOUT; timeout_ns <= 0 waits without limit).
 * Requests from many threads are batched by the serving loop, admitted
 * against the context's cache budget, built on the device and kept in an
 * LRU relation cache.  On success *out pins the cache entry until
 * gale_release.  EBUSY if the budget is pinned by other views, ENOMEM if one
 * cluster alone exceeds the budget, EINVAL on a bad id or mask.
 */
gale_status gale_request(gale_ctx *ctx, int32_t cluster_id, uint32_t mask, int64_t timeout_ns, gale_view *out);

/* Serving execution forms. */
enum {
    GALE_SERVE_LOOP = 0,   /* device-resident request loop (default when some size bin fits it) */
    GALE_SERVE_BATCH = 1,  /* the leader launches the batched kernels for each batch of admitted requests */
    GALE_SERVE_SINGLE = 2  /* one kernel launch per request, one at a time (the baseline form) */
};

/* Choose the serving form, the loop's idle exit (microseconds, 0 = default
 * 20000), the most CTAs the device loop may occupy (loop_ctas, 0 = as many
 * as fit on the device; a cap lets the loops of several loaded meshes stay
 * resident side by side) and the proactive prefetch depth (prefetch = m: a
 * request for cluster k also queues clusters k+1 .. k+m with the same mask
 * unless cached or queued, the paper's leader building the requested segment
 * together with the following ones, Section 4.5; prefetched entries pin
 * nothing, are admitted only while no request waits and only into free
 * cache space, never evicting, and are dropped when the budget is full)
 * before the first gale_request of the context;
 * EBUSY afterwards, EINVAL for an unknown mode, a negative cap or depth, or when no
 * size bin fits the loop.  The loop builds every cluster under the
 * cluster's own working-memory plan at one block size, and serves the size
 * bins whose clusters each fit one CTA; requests for clusters of the other
 * bins (global-scratch bins) are built by batched launches beside it.  A
 * thread waiting in gale_request advances admission, publication and
 * completion itself whenever the leader thread has not lately, so requests
 * progress even while consumer threads occupy every host core. */
gale_status gale_serve_configure(gale_ctx *ctx, int32_t mode, int64_t idle_us, int32_t loop_ctas, int32_t prefetch);

/* Unpin a view from gale_request; its entry becomes evictable.  The view's
 * handle names its pin, not the entry: releasing a view twice, or after its
 * lease ran out, returns ENOTFOUND and touches nothing. */
gale_status gale_release(gale_ctx *ctx, gale_view *view);

/* Lease of the pins that later gale_request calls hand out: a view not
 * released within lease_ns nanoseconds is unpinned by the serving leader
 * (its entry becomes evictable, leases_expired counts it), so a consumer
 * thread that dies holding views cannot keep the budget pinned.  0 (the
 * default) = no limit.  A consumer must not read a view after its lease. */
gale_status gale_serve_set_lease(gale_ctx *ctx, int64_t lease_ns);

/* Serving counters (requests, hits, builds, evictions, ...). */
gale_status gale_serve_stats_get(gale_ctx *ctx, gale_serve_stats *out);

/* Canonical <-> input ids: vperm[c] = input id of canonical vertex c
 * (int32[nv]), tperm[c] = input index of canonical tet c (int32[nt]).  Either
 * pointer may be NULL.  Host memory. */
gale_status gale_get_permutations(gale_ctx *ctx, int32_t *vperm, int32_t *tperm);

/* Interval arrays I_V and I_T (int64[nclusters+1] each, host) and the exact
 * per-cluster sizes (int64[nclusters*5]: VT, VV, edges, ET, TT entries; NULL
 * allowed; zeros in a host-only context). */
gale_status gale_get_intervals(gale_ctx *ctx, int64_t *I_V, int64_t *I_T, int64_t *sizes);

/* Canonical rows (int32[nt*4], host) in canonical tet order. */
gale_status gale_get_rows(gale_ctx *ctx, int32_t *rows);

/* Working set of cluster k: T_ex(k) and halo(k) as ascending canonical tet
 * ids (caller buffers; *n_ext / *n_halo in: capacity, out: count). */
gale_status gale_get_working_set(gale_ctx *ctx, int32_t k, int32_t *ext, int64_t *n_ext, int32_t *halo,
                                 int64_t *n_halo);

gale_status gale_get_info(gale_ctx *ctx, gale_info *out);

/*
 * Edge and triangle enumeration (Section 4.3, "Initialization": E and F are
 * enumerated on the CPU, with interval arrays I_E and I_F; only when the
 * analysis needs edges or triangles).  An edge (u, w), u < w, or a triangle
 * (a, b, c), a < b < c, in canonical vertex ids, belongs to the segment of
 * its lowest vertex; segment k's simplices have the global ids
 * [I_E[k], I_E[k+1]) (resp. I_F).  Within a segment they are numbered
 *   GALE_ENUM_SORTED            lexicographically (the (u, w) order of the
 *                               edges of the ET relation), or
 *   GALE_ENUM_FIRST_APPEARANCE  by first appearance while the segment's
 *                               tetrahedra are visited in canonical order,
 *                               each tetrahedron's vertex combinations in
 *                               combination order (the numbering of the
 *                               paper's worked example FE(f5) = {e2, e6, e9}).
 * Host work, on host-only contexts too; replaces an earlier enumeration.
 * On a device context with ET preconditioned, GALE_ENUM_SORTED is built on
 * the GPU instead: only I_E and I_F come to the host, and the lists stay in
 * device memory (held for gale_build_coboundary) until gale_get_enumeration
 * copies them to the caller or gale_boundary makes its host copy.
 */
enum { GALE_ENUM_SORTED = 0, GALE_ENUM_FIRST_APPEARANCE = 1 };
gale_status gale_enumerate(gale_ctx *ctx, int32_t order);

/* The enumeration (host memory; any pointer may be NULL): counts[2] = edges,
 * triangles; edges int32[2 nE] (u, w); I_E int64[K+1]; faces int32[3 nF]
 * (a, b, c); I_F int64[K+1].  Lists still on the device are copied straight
 * into edges / faces (as gale_copy_to_host does).  ENOTFOUND before
 * gale_enumerate; ECUDA if a device copy fails. */
gale_status gale_get_enumeration(gale_ctx *ctx, int64_t *counts, int32_t *edges, int64_t *I_E, int32_t *faces,
                                 int64_t *I_F);

/* Boundary relations, per simplex, by lookup in the enumeration within the
 * owning segment's interval (Section 4.4):
 *   GALE_REL_FE  triangle ids -> 3 edge ids each: (a,b), (a,c), (b,c)
 *   GALE_REL_TE  canonical tet ids -> 6 edge ids each, combination order
 *                (a,b), (a,c), (a,d), (b,c), (b,d), (c,d)
 *   GALE_REL_TF  canonical tet ids -> 4 triangle ids each: (a,b,c),
 *                (a,b,d), (a,c,d), (b,c,d)
 * ids: HOST int64[n]; out: HOST int32[width * n].  The first call after a
 * device enumeration copies the lists to the host and builds the lookup
 * index.  EINVAL on an id out of range, ENOTFOUND before gale_enumerate,
 * ENOMEM if the host copy or index cannot be allocated. */
enum { GALE_REL_FE = 1, GALE_REL_TE = 2, GALE_REL_TF = 3 };
gale_status gale_boundary(gale_ctx *ctx, int32_t relation, const int64_t *ids, int64_t n, int32_t *out);

/*
 * Coboundary relations VE, VF, EF and FT of the whole mesh, in the ids of
 * the enumeration (gale_enumerate first), built on the GPU (Section 4.4:
 * coboundary relations are delegated to the GPU; Section 5 evaluates VE, VF,
 * EF and FT).  Rows ascending:
 *   GALE_CB_VE  rows = vertices (canonical ids): the edges containing v
 *   GALE_CB_VF  rows = vertices: the triangles containing v
 *   GALE_CB_EF  rows = edges (enumeration ids): the triangles containing e
 *   GALE_CB_FT  rows = triangles: the canonical tets containing f
 * The pass reads only the enumeration and the canonical tet rows (the bulk
 * arrays are left alone).  In vertex-tuple order a row's entries come as one
 * contiguous range (VE(v): the edges with lower vertex v; EF(e): the
 * triangles whose first two vertices are e; VF(v): the triangles with lowest
 * vertex v) and the rest scattered from the simplices that hold the row's
 * simplex elsewhere (edge (a, b) into VE(b); triangle (a, b, c) into
 * EF(a, c), EF(b, c), VF(b), VF(c); a tet into FT of its faces), found
 * through a per-vertex index of the enumeration built on the device once per
 * enumeration; every row is then sorted by id.  out receives, per relation
 * in the order VE, VF, EF, FT, the row count, the value count and DEVICE
 * pointers to int32 offsets[rows+1] and values, library-owned and valid
 * until the next call or gale_destroy.  EINVAL if the enumeration has 2^31
 * or more edges or triangles (or a relation 2^31 or more entries), ENOTFOUND
 * before gale_enumerate, EDEVICE if a lookup failed.  FT takes two slots
 * per triangle; on a non-manifold mesh (a triangle in three or more tets:
 * known at load when GALE_TT is preconditioned, else found when the slots
 * overflow, and the pass then runs again) it counts each triangle's tets,
 * places them by cursors and sorts the rows. */
enum { GALE_CB_VE = 1, GALE_CB_VF = 2, GALE_CB_EF = 4, GALE_CB_FT = 8 };
typedef struct {
    int64_t rows[4];
    int64_t len[4];
    const int32_t *off[4];
    const int32_t *val[4];
} gale_coboundary;
gale_status gale_build_coboundary(gale_ctx *ctx, uint32_t which, gale_coboundary *out);

/* Tuning: threads per block of the producer kernels (a multiple of 32 in
 * [64, 1024]; 0 = one thread per own vertex of the largest cluster of each
 * size bin) and CTAs per SM of the persistent grid (0 = as many as fit). */
gale_status gale_set_tuning(gale_ctx *ctx, int32_t threads, int32_t ctas_per_sm);

/* Several small clusters per CTA (no counterpart in the paper, which runs a
 * fixed 32 threads per segment; Section 4.6, Appendix A): every size bin of
 * whole clusters in shared memory (not global-scratch, per-item or cut-
 * cluster bins, nor bins of parts) whose plan at team_threads fits `teams`
 * times in one CTA's shared memory is launched, in batched builds, with
 * `teams` teams of team_threads threads per CTA, each team taking clusters
 * on its own with barriers of its own.  team_threads: a multiple of 32;
 * teams: 2..15 with team_threads * teams <= 512; teams = 0 turns it off.
 * gale_get_bins reports it; gale_autotune also tries it.  The per-cluster
 * form, serving and the allocation-free build still run one cluster per
 * CTA under the same plan.  EINVAL on bad sizes. */
gale_status gale_set_teams(gale_ctx *ctx, int32_t team_threads, int32_t teams);

/* Size bins: for each bin (up to max_bins) nine int32 values - members,
 * threads per CTA, bytes of per-CTA working memory, CTAs per SM, persistent
 * grid size, 1 if the working memory is global scratch (too large for
 * shared memory) else 0, 1 if every member runs under its own shared-memory
 * plan (the largest clusters, whose plans do not merge) else 0, and the
 * number of members that are parts of cut clusters (gale_mesh_desc
 * part_vertices), or -1 for a bin of cut clusters themselves, which batched
 * builds skip (they build the parts) and the per-cluster form, serving and
 * gale_build_clusters_noalloc use, and the teams per CTA of its batched
 * launches (0: one cluster per CTA; gale_set_teams) - into
 * out[9*i .. 9*i+8].  Returns the number of bins in *nbins. */
gale_status gale_get_bins(gale_ctx *ctx, int32_t *out, int32_t max_bins, int32_t *nbins);

/* Members of the size bins: the work item ids of bin 0, then bin 1, ...
 * (K + nparts ids in all, gale_info; the counts per bin are gale_get_bins'
 * first values), each bin in its launch order (largest working set first).
 * Ids below K are clusters; id K + p is part p (parts are numbered cluster
 * by cluster, in vertex order).  out: K + nparts int32. */
gale_status gale_get_bin_members(gale_ctx *ctx, int32_t *out);

/* Autotune the batched form.  For every size bin, the bin's clusters are
 * built alone (relations in mask, outputs into the bulk arrays) with every
 * candidate block size - 128, 256, 384, 512, 768 and 1024 threads whose
 * working memory fits - and every CTA-per-SM count that fits, each timed
 * over reps launches (0 = 2) with CUDA events after one untimed launch; the
 * fastest pair is kept for the bin (gale_get_bins reports it) and captured
 * full builds are dropped so the next one captures the choice.  best_ms
 * (optional, max_bins entries): the chosen time per bin.  A later
 * gale_set_tuning call replaces the choice. */
gale_status gale_autotune(gale_ctx *ctx, uint32_t mask, int32_t reps, float *best_ms, int32_t max_bins);

/* The stream of the context (cudaStream_t). */
void *gale_stream(gale_ctx *ctx);

/* Number of kernel launches the last gale_build_clusters enqueued. */
int64_t gale_last_launch_count(gale_ctx *ctx);

void gale_destroy(gale_ctx *ctx);

/* Thread-local message of the last failing call on this thread. */
const char *gale_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GALE_H */
