// Internal layout shared by the host runtime (gale_*.cpp) and the kernels
// (gale_kernels.cu).  Not part of the public ABI.
#pragma once

#include <stdint.h>
#include <stddef.h>

#include <vector>

#if defined(__CUDACC__)
#define GALE_HD __host__ __device__
#else
#define GALE_HD
#endif

namespace gale {

// ---------------------------------------------------------------------------
// Cluster working set ("block"), one per cluster, contiguous in device memory
// and 16-byte aligned.  All sections are int32 words; every section starts on
// a multiple of 4 words so the block can be moved with 16-byte vector loads
// or one bulk copy.
//
//   [0, 12)               header (BlockHdr)
//   [12, 12 + a4(nv_loc)) vmap: canonical id of each local vertex
//   next a4(n_ext+n_halo) tmap: canonical ids of the external tets (ascending,
//                         all below the cluster's first internal tet) then of
//                         the halo tets (ascending)
//   next a4(2 * n_tot)    rows: 4 x uint16 local vertex ids per tet (ascending
//                         within the row), tets in local order
//                         [external | internal | halo]
//   next a4(ceil(n_bnd/2)) bnd: uint16 internal-tet indices (0 = first
//                         internal tet) of the internal tets (a, b, c, d)
//                         whose face (b, c, d) has no own vertex, ascending
//
// Local vertex ids [0, nv_nb) are the vertices of the external and internal
// tets in canonical order (so local order equals canonical order there);
// they include the cluster's own vertices as the interval
// [own_lo, own_lo + nv_own) = canonical [v_base, v_base + nv_own).  Ids
// [nv_nb, nv_loc) are vertices that only halo tets use.  Local tet i maps to
//   i <  n_ext                tmap[i]
//   i <  n_ext + n_own        t_base + (i - n_ext)
//   otherwise                 tmap[i - n_own]
// and since external tets precede the internal ones in canonical order, the
// local order of [external | internal] is canonical order too.  n_bnd counts
// the internal tets (a, b, c, d) whose face (b, c, d) has no own vertex.
//
// Part blocks (part != 0).  A cluster too large for one CTA's shared memory
// is also cut into parts: contiguous ranges of its own vertices, each built
// by its own CTA straight into the cluster's output arrays.  A part's own
// vertices are its range; its external tets are the cluster's external tets
// that touch the range, and its internal tets are the cluster's internal tets
// that touch the range, in canonical order (not a contiguous id range, so
// their ids follow the halo ids in tmap: tmap has n_ext + n_halo + n_own
// words).  The part builds VT, VV and ET of its own vertices and the TT rows
// of the internal tets whose lowest vertex is its own; n_bnd counts those.
// ---------------------------------------------------------------------------
struct BlockHdr {
    int32_t n_ext, n_own, n_halo, nv_loc;
    int32_t own_lo, nv_own, t_base, v_base;
    int32_t nv_nb, n_bnd, part, pad1;  // part: 0, or 1 + the part's index
};
static_assert(sizeof(BlockHdr) == 48, "header is 12 words");
constexpr int kHdrWords = 12;

GALE_HD inline int64_t a4(int64_t x) { return (x + 3) & ~int64_t(3); }
// n_xmap: extra tmap words (a part block's internal tet ids; 0 otherwise)
GALE_HD inline int64_t blk_words(int32_t nv_loc, int32_t n_ext, int32_t n_own, int32_t n_halo, int32_t n_bnd,
                                 int32_t n_xmap = 0) {
    return kHdrWords + a4(nv_loc) + a4(int64_t(n_ext) + n_halo + n_xmap) + a4(2 * (int64_t(n_ext) + n_own + n_halo)) +
           a4((int64_t(n_bnd) + 1) / 2);
}
GALE_HD inline int64_t blk_tmap_off(int32_t nv_loc) { return kHdrWords + a4(nv_loc); }
GALE_HD inline int64_t blk_rows_off(int32_t nv_loc, int32_t n_ext, int32_t n_halo, int32_t n_xmap = 0) {
    return kHdrWords + a4(nv_loc) + a4(int64_t(n_ext) + n_halo + n_xmap);
}
GALE_HD inline int64_t blk_bnd_off(int32_t nv_loc, int32_t n_ext, int32_t n_own, int32_t n_halo, int32_t n_xmap = 0) {
    return blk_rows_off(nv_loc, n_ext, n_halo, n_xmap) + a4(2 * (int64_t(n_ext) + n_own + n_halo));
}

// Largest local id space a block can address (uint16 local ids).
constexpr int32_t kMaxLocal = 65535;

// Per-cluster sizes (entries) found by the counting pass.
enum { SZ_VT = 0, SZ_VV = 1, SZ_E = 2, SZ_ET = 3, SZ_TT = 4, SZ_N = 5 };
// counting pass only, one past the sizes: 1 when the cluster's TT rows take
// the general pass (a triangle of the cluster lies in three or more tets)
constexpr int SZ_GENERAL = SZ_N;

// Relation mask bits (same values as the public GALE_* bits).
enum : uint32_t { R_VT = 1u, R_VV = 2u, R_ET = 4u, R_TT = 8u };

// One unit of kernel work: a cluster, which relations, where its block is,
// and where each output array of this cluster starts (NULL = not built).
struct WorkItem {
    int32_t k;
    uint32_t mask;
    int64_t blk;  // word offset of the cluster's block
    int32_t *vt_off, *vt_val, *vv_off, *vv_val;
    int32_t *eu_off, *e_w, *et_off, *et_val;
    int32_t *tt_off, *tt_val;
};
static_assert(sizeof(WorkItem) == 96, "work item is 96 bytes");

// One part of a cut cluster (see the block layout above).  Work items are
// numbered clusters first, then parts: item K + p is part p.  A batched
// build lists a cut cluster's parts in order in place of the cluster, so the
// output placement of consecutive parts is the cluster's own: each part's
// offset arrays hold its own entries and the last part's also the final
// one.  The b_* fields are the cluster-level values at the part's start.
struct PartInfo {
    int32_t k;        // the cluster
    int32_t x0;       // first own vertex, relative to the cluster's
    int32_t nvo;      // own vertices
    int32_t last;     // 1 for the cluster's last part
    int32_t b_vt, b_vv, b_e, b_et;  // VT, VV, owned-edge and ET entries of the earlier parts
    int32_t b_tt;     // TT entries of the earlier parts
    int32_t b_to;     // TT rows (internal tets) of the earlier parts
    int32_t n_rows;   // internal tets whose lowest vertex is the part's (its TT rows)
    int32_t tt_total; // the cluster's TT entries
    int32_t n_own_c;  // the cluster's internal tets
    int32_t t_base_c; // the cluster's first internal tet
    int32_t pad[2];
};
static_assert(sizeof(PartInfo) == 64, "part record is 64 bytes");

// Per-cluster facts the host learns at load time, used for bins and bounds.
struct ClusterStat {
    int32_t n_ext, n_own, n_halo, nv_loc, nv_own;
    int32_t n_vt;     // incidences of own vertices in [external | internal]
    int32_t max_deg;  // largest VT row
    int32_t nv_nb;    // local vertices of the external and internal tets
    int32_t n_bnd;    // internal tets whose face opposite their lowest vertex has no own vertex
    int32_t max_up;   // most distinct upper neighbours of an own vertex
    int32_t n_e;      // edges whose lower endpoint is an own vertex
    int32_t xmap;     // extra tmap words of the block (a part's internal tet ids; 0 for a cluster)
};

// Capacities a launch is planned for (maxima over the clusters it serves).
struct Caps {
    int32_t blk_words;  // largest block
    int32_t nv_own;     // largest own vertex count
    int32_t n_vt;       // largest sum of VT rows
    int32_t n_own;      // largest internal tet count
    int32_t nv_loc;     // largest local vertex count
    int32_t nv_nb;      // largest neighbour-universe size (bitmap bits)
    int32_t max_deg;    // largest VT row
    int32_t max_vv;     // largest sum of VV rows   (0 in counting plans)
    int32_t max_e;      // largest owned edge count
    int32_t max_etv;    // largest sum of ET rows   (0 in counting plans)
    int32_t max_tt;     // largest sum of TT rows   (0 in counting plans)
    int32_t max_up;     // most upper neighbours of an own vertex
    int32_t hcap;       // boundary-face hash capacity (power of two)
    int32_t n_tot;      // largest tet count of a block (external + internal + halo)
    int32_t n_star;     // largest external + internal tet count
};

// Byte offsets of the shared-memory regions of one CTA (all 16-aligned).
// Two regions are reused from phase to phase:
//   r2: VV and upper-endpoint staging, then the per-edge tet masks (which
//       end up holding the ET row offsets);
//   r1: VT per-warp counters and lane masks; then the neighbour bitmaps and
//       their rank prefixes; then ET staging; then the boundary-face hash,
//       the TT counts and the TT staging.
struct SmemPlan {
    int32_t threads;
    int32_t W;          // row stride (words, odd) of the neighbour bitmaps
    int32_t nch;        // 32-tet chunks of the longest VT row
    int32_t pad;        // per-warp counter row length (even)
    int32_t scan;       // scan scratch (3 x 33 words)
    int32_t blk;        // int32[blk_words] the cluster's block (bulk copy)
    int32_t vt_off;     // int32[nv_own+1]
    int32_t vt_list;    // uint16[n_vt]
    int32_t c_vv;       // int32[nv_own+1] VV row offsets
    int32_t c_e;        // int32[nv_own+1] first owned edge of each own vertex
    int32_t nbr;        // uint16[4*n_own] TT links
    int32_t jpos;       // uint8 (or uint16 when jpos16)[4*n_star]: position of each
                        // (tet, own slot) in that vertex's VT row
    int32_t jpos16;     // 1: VT rows may exceed 256 entries, positions are 16-bit
    int32_t r2;         // uint16[max_vv] VV staging | uint32[max_e*nch] edge masks
    int32_t st_w;       // uint16[max_e] upper-endpoint staging (inside r2)
    int32_t r1;         // see above
    int32_t mk;         // phase B lane masks (inside r1)
    int32_t pre;        // uint8[nv_own*W] rank prefixes (inside r1)
    int32_t tcnt;       // int32[n_own+1] TT counts (inside r1)
    int32_t st_tt;      // uint16[max_tt] TT staging (inside r1)
    int32_t total;      // bytes
    Caps caps;
};

// Device error word bits.
enum : int32_t {
    ERR_CAPACITY = 1,      // a cluster exceeded the capacities of its launch
    ERR_NONMANIFOLD = 2,   // a triangle is shared by more than two tets
    ERR_HASH_FULL = 4,     // face hash probe ran past its capacity
    ERR_BAD_ITEM = 8,      // a work item referenced a bad cluster
    ERR_TIMEOUT = 16,      // a bounded device wait ran out
    ERR_BAD_BLOCK = 32,    // a block broke an invariant of its layout
};

SmemPlan plan_smem(const Caps &c, int threads);
// Capacities of one cluster or part; staging capacities come from the exact
// sizes of the counting pass (sizes == nullptr: a counting plan, no staging).
Caps caps_of(const ClusterStat &s, const int64_t *sizes);
// Shared memory a build plan of this working set would take at the given
// block size, with its staging sized from estimates (the counting pass has
// not run yet): used to decide which clusters to cut into parts.
int64_t estimate_smem(const ClusterStat &s, int threads);

// Size bins a context may have (one ticket counter each in the build and
// serving paths).
constexpr int kMaxBins = 64;

// A cluster is cut into parts of about kPartVertices own vertices when the
// estimate exceeds kCutBytes (both overridable at load time).
constexpr int32_t kPartVertices = 256;
constexpr int64_t kCutBytes = 160 * 1024;
// ... and into twice as many parts while some part's estimate exceeds this.
constexpr int64_t kPartFitBytes = 200 * 1024;

// Kernel launchers (gale_kernels.cu).  All asynchronous on `stream`.
struct DevMesh {
    const int32_t *blocks;      // all cluster blocks, then all part blocks
    const int64_t *blk_off;     // [K+NP+1] word offset of each block
    const int32_t *I_V;         // [K+1]
    const int32_t *I_T;         // [K+1]
    int32_t K;
    int32_t NP;                 // parts of cut clusters (work items K .. K+NP-1)
    const PartInfo *parts;      // [NP]
    int32_t *tt_pos;            // [nt] per internal tet of a cut cluster: its TT row's
                                // offset in the cluster (the counting pass writes
                                // the row lengths here first)
    int32_t *tt_general;        // [K] the counting pass writes 1 where the cluster's TT
                                // rows take the general pass (non-manifold), else 0
};

// Persistent launch over n clusters: ids[i] (count pass) or items[order[i]]
// (build).  One CTA per cluster at a time.
// gscratch: NULL runs the cluster in dynamic shared memory; otherwise each
// CTA uses the slice gscratch + blockIdx.x * plan.total of global memory.
// mask: the relations the context is preconditioned for (TT sizes only
// when it holds R_TT).
// plans (non-NULL): every cluster k runs under its own plan plans[k] (device
// memory), and `plan` only gives the launch's block size and the dynamic
// shared memory (the largest of the plans); never with gscratch.
int launch_count_pass(const DevMesh &m, const SmemPlan &plan, const int32_t *ids, int32_t n, int64_t *sizes_out,
                      int32_t *err, int32_t *ticket, int grid, void *stream, char *gscratch, uint32_t mask,
                      const SmemPlan *plans = nullptr);
// Output placement for n listed clusters (three launches).  bsum: device
// scratch of bases_scratch_words(n) int64 words.
int bases_scratch_words(int32_t n);
int launch_bases(const DevMesh &m, const int32_t *ids, int32_t n, const int64_t *sizes, uint32_t mask,
                 const WorkItem *arrays_base, WorkItem *items, int64_t *totals_out, int64_t *bsum, void *stream);
// teams > 0: several clusters per CTA, one team of plan.threads threads each
// (`teams` of them per CTA, each with plan.total bytes of shared memory);
// never with plans or gscratch.
int launch_build(const DevMesh &m, const SmemPlan &plan, const WorkItem *items, const int32_t *order, int32_t n,
                 int32_t *err, int32_t *ticket, int grid, void *stream, char *gscratch,
                 const SmemPlan *plans = nullptr, int teams = 0);
// One launch, one CTA, one work item (the per-cluster baseline form).
int launch_build_one(const DevMesh &m, const SmemPlan &plan, const WorkItem *items, int32_t index, int32_t *err,
                     void *stream, char *gscratch);
// Ring of the device-resident serving loop (all host pointers are mapped
// host memory seen through device addresses).
struct ServeRing {
    const WorkItem *items;        // [cap]
    const long long *tail;        // tickets published so far
    long long *done;              // [cap] last ticket completed in each slot
    const int *stop;              // non-zero: loop returns
    unsigned long long *next;     // device memory: next ticket to claim
    int32_t cap;
    int32_t pad;
    unsigned long long idle_ns;   // a CTA returns after this long without work
    long long *times;             // [2 cap] device clock (ns) at a ticket's claim and completion
};
// plans: the plan each cluster is built under (device memory, indexed by
// cluster id); `plan` gives the block size and the dynamic shared memory.
int launch_serve(const DevMesh &m, const SmemPlan &plan, const SmemPlan *plans, const ServeRing &ring, int32_t *err,
                 int grid, void *stream);
int serve_ctas_per_sm(const SmemPlan &plan);

int kernel_smem_limit();
int max_ctas_per_sm(const SmemPlan &plan, bool spill, bool per_item = false);
// CTAs per SM of a team launch (0 if it cannot launch)
int max_ctas_per_sm_teams(const SmemPlan &plan, int teams);
// Sets the dynamic shared memory limit of the cluster kernels to smem
// (clamped to dynamic_smem_limit()); false if the runtime refused.
bool prepare_kernels(int smem);
int dynamic_smem_limit();
int device_sm_count();

}  // namespace gale
