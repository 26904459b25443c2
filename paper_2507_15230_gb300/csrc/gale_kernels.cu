// Producer kernels: per-cluster VT, VV, ET and TT as canonical sorted CSR.
//
// One CTA builds one cluster at a time (persistent CTAs take clusters from a
// ticket counter; the per-cluster baseline launches one CTA per cluster).
// The rows of the cluster's working set - its internal tets, its external
// tets T_ex and its face halo (Section 4.3, "Initialization"), as 16-bit
// local rows - arrive in shared memory by one bulk copy, and every relation
// is built there.  Each phase spreads its work evenly over all threads of the
// block (over tets, bitmap words, VT incidences, edges or internal tets), so
// the block size is free of the cluster's vertex count; the outputs leave
// through shared-memory staging with one thread per element (coalesced),
// except TT's rows of at most four entries, stored straight out.
//
//  B. VT (Section 4.6 / Algorithm 1: iterate the segment's tets and test
//     each vertex against the segment interval).  Each warp takes a
//     contiguous chunk of the tets (which are in canonical order) and counts
//     its incidences per own vertex; a prefix across warps gives every
//     (warp, vertex) its first slot, and within a warp the lanes holding the
//     same vertex are ranked by a 32-bit lane mask.  Rows come out ascending
//     with no sort.  (The paper's atomicPush, Algorithm 2, fills rows in
//     arbitrary order.)
//  C. VV and the edges (x, w), x < w, that an own vertex x owns:
//     - C1, per tet: the other vertices of every tet of VT(x) are ORed into
//       a bitmap of x over the cluster's vertex universe; local order is
//       canonical order, so the bitmap read in bit order is VV(x), sorted and
//       deduplicated, and its bits above x are the upper endpoints w;
//     - C2, per bitmap word: one block scan of the word popcounts places
//       every VV row and every edge; each word keeps the rank of its first
//       upper bit within its vertex, so an edge's index is one popcount away;
//     - C3, per VT incidence (x, j-th tet of VT(x)): bit j is set in the tet
//       mask of each edge (x, w) of that tet; a mask read in bit order is
//       ET(x, w), ascending;
//     - C5, per internal tet (a, b, c, d): the AND of the masks of two edges
//       (a, w1), (a, w2) holds the two tets of the face (a, w1, w2); the face
//       (b, c, d) is matched the same way inside VT(b) when b is own;
//     - C4, per edge: the mask bits become the ET rows.
//  D. TT (Table 1; the paper gives no kernel for it) for the faces (b, c, d)
//     of internal tets (a, b, c, d) with no own vertex: a small
//     open-addressing hash of those faces is probed with the faces of the
//     halo tets.
//  E. TT rows from the four face links, sorted by canonical id.  A face with
//     a second partner (a triangle in three or more tets) marks the cluster
//     instead, whose rows then come from E', a general pass over the block
//     (compiled into every kernel but the hot shared-memory one: the
//     counting pass reports such clusters and the host runs them from
//     per-item bins).  Parts of cut clusters report it as an error.
//
// The counting mode runs the same passes without writes and returns the
// exact sizes the host uses to place outputs and to admit cache entries.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "gale_internal.h"

namespace gale {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kWaitLimit = 1 << 22;  // polls of the block copy's barrier before giving up

struct Smem {
    int32_t *scan;
    int32_t *blk;
    int32_t *vt_off;
    uint16_t *vt_list;
    int32_t *c_vv, *c_e;
    uint16_t *nbr;
    uint8_t *jpos;
    uint32_t *emask;  // r2
    uint16_t *st_v;   // r2
    uint16_t *st_w;   // r2
    uint16_t *cw;     // r1 (phase B)
    uint32_t *mk;     // r1 (phase B)
    uint32_t *bm;     // r1 (phase C)
    uint8_t *pre;     // r1 (phase C)
    uint16_t *st_et;  // r1 (phase C4)
    uint32_t *hash;   // r1 (phase D)
    int32_t *tcnt;    // r1 (phases D, E)
    uint16_t *st_tt;  // r1 (phase E)
};

__device__ __forceinline__ Smem carve(char *base, const SmemPlan &p) {
    Smem s;
    s.scan = reinterpret_cast<int32_t *>(base + p.scan);
    s.blk = reinterpret_cast<int32_t *>(base + p.blk);
    s.vt_off = reinterpret_cast<int32_t *>(base + p.vt_off);
    s.vt_list = reinterpret_cast<uint16_t *>(base + p.vt_list);
    s.c_vv = reinterpret_cast<int32_t *>(base + p.c_vv);
    s.c_e = reinterpret_cast<int32_t *>(base + p.c_e);
    s.nbr = reinterpret_cast<uint16_t *>(base + p.nbr);
    s.jpos = reinterpret_cast<uint8_t *>(base + p.jpos);
    s.emask = reinterpret_cast<uint32_t *>(base + p.r2);
    s.st_v = reinterpret_cast<uint16_t *>(base + p.r2);
    s.st_w = reinterpret_cast<uint16_t *>(base + p.st_w);
    s.cw = reinterpret_cast<uint16_t *>(base + p.r1);
    s.mk = reinterpret_cast<uint32_t *>(base + p.mk);
    s.bm = reinterpret_cast<uint32_t *>(base + p.r1);
    s.pre = reinterpret_cast<uint8_t *>(base + p.pre);
    s.st_et = reinterpret_cast<uint16_t *>(base + p.r1);
    s.hash = reinterpret_cast<uint32_t *>(base + p.r1);
    s.tcnt = reinterpret_cast<int32_t *>(base + p.tcnt);
    s.st_tt = reinterpret_cast<uint16_t *>(base + p.st_tt);
    return s;
}

// ---- bulk copy into shared memory, completion on an mbarrier ----
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    // order this CTA's earlier generic accesses of dst before the async write
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
// bulk prefetch of [p, p + bytes) into L2 (16-byte aligned, multiple of 16)
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < kWaitLimit; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ uint32_t vtx(uint2 r, int s) {
    uint32_t w = (s < 2) ? r.x : r.y;
    return (s & 1) ? (w >> 16) : (w & 0xffffu);
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Who builds a cluster: the whole CTA, or a team - a warp-aligned slice of
// it with a named barrier of its own (several small clusters per CTA).
struct BlockTeam {
    __device__ __forceinline__ int nt() const { return blockDim.x; }
    __device__ __forceinline__ int tid() const { return threadIdx.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ int sync_or(int p) const { return __syncthreads_or(p); }
};
struct SliceTeam {
    int n;    // threads (a multiple of 32)
    int t;    // this thread's index in the team
    int bar;  // named barrier id (1..15; 0 is __syncthreads')
    __device__ __forceinline__ int nt() const { return n; }
    __device__ __forceinline__ int tid() const { return t; }
    __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(n) : "memory"); }
    __device__ __forceinline__ int sync_or(int p) const {
        int r;
        asm volatile(
            "{\n\t.reg .pred pin, pout;\n\tsetp.ne.s32 pin, %1, 0;\n\t"
            "bar.red.or.pred pout, %2, %3, pin;\n\tselp.s32 %0, 1, 0, pout;\n\t}"
            : "=r"(r)
            : "r"(p), "r"(bar), "r"(n)
            : "memory");
        return r;
    }
};

// Exclusive scan of one value per thread over the team (any multiple of 32
// threads up to 1024); scr needs 33 words.  Two team barriers.
template <class Team>
__device__ __forceinline__ int block_scan_thread(const Team &tm, int v, int32_t *scr, int *total) {
    const int nw = tm.nt() >> 5;
    const int lane = tm.tid() & 31, warp = tm.tid() >> 5;
    const int incl = warp_incl_scan(v, lane);
    if (lane == 31) scr[warp] = incl;
    tm.sync();
    if (warp == 0) {
        const int w = lane < nw ? scr[lane] : 0;
        const int wi = warp_incl_scan(w, lane);
        if (lane < nw) scr[lane] = wi - w;
        if (lane == 31) scr[32] = wi;
    }
    tm.sync();
    *total = scr[32];
    return scr[warp] + incl - v;
}

// Exclusive scans of three values per thread over the team, in place;
// totals to t[0..2].  scr needs 99 words.  Ends synced.
template <class Team>
__device__ __forceinline__ void block_scan3(const Team &tm, int &a, int &b, int &c, int32_t *scr, int *t) {
    const int nw = tm.nt() >> 5;
    const int lane = tm.tid() & 31, warp = tm.tid() >> 5;
    const int ia = warp_incl_scan(a, lane), ib = warp_incl_scan(b, lane), ic = warp_incl_scan(c, lane);
    if (lane == 31) {
        scr[warp] = ia;
        scr[33 + warp] = ib;
        scr[66 + warp] = ic;
    }
    tm.sync();
    if (warp == 0) {
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int w = lane < nw ? scr[33 * s + lane] : 0;
            const int wi = warp_incl_scan(w, lane);
            if (lane < nw) scr[33 * s + lane] = wi - w;
            if (lane == 31) scr[33 * s + 32] = wi;
        }
    }
    tm.sync();
    t[0] = scr[32];
    t[1] = scr[65];
    t[2] = scr[98];
    a = scr[warp] + ia - a;
    b = scr[33 + warp] + ib - b;
    c = scr[66 + warp] + ic - c;
    tm.sync();
}

// p[0 .. n) = v over the team, 16 bytes a store (p is 16-byte aligned: every
// region of the plan is).
template <class Team>
__device__ __forceinline__ void fill_words(const Team &tm, uint32_t *p, int n, uint32_t v) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
    const int n4 = n >> 2;
    const uint4 v4 = make_uint4(v, v, v, v);
    for (int i = tm.tid(); i < n4; i += tm.nt()) q[i] = v4;
    for (int i = 4 * n4 + tm.tid(); i < n; i += tm.nt()) p[i] = v;
}

// Length of each thread's contiguous range when n items are split over the
// team: odd, so that neighbouring threads start in different banks.
template <class Team>
__device__ __forceinline__ int range_len(const Team &tm, int n) {
    const int per = (n + tm.nt() - 1) / tm.nt();
    return per > 1 ? (per | 1) : per;
}

// dst[j] = f(j) for j < n over the team, four loads in flight per thread
// before their stores (the values come through L2 from the block's maps).
template <class Team, typename F>
__device__ __forceinline__ void copy_out(const Team &tm, int32_t *__restrict__ dst, int n, F f) {
    const int NT = tm.nt();
    int j = tm.tid();
    for (; j + 3 * NT < n; j += 4 * NT) {
        const int32_t a = f(j), b = f(j + NT), c = f(j + 2 * NT), d = f(j + 3 * NT);
        dst[j] = a;
        dst[j + NT] = b;
        dst[j + 2 * NT] = c;
        dst[j + 3 * NT] = d;
    }
    for (; j < n; j += NT) dst[j] = f(j);
}

// Exclusive scan in place of a[0..n); returns the total.  Ends synced.
template <class Team>
__device__ int block_scan_array(const Team &tm, int32_t *a, int n, int32_t *scr) {
    const int per = range_len(tm, n);
    const int b = min(n, tm.tid() * per);
    const int e = min(n, b + per);
    int s = 0;
    for (int i = b; i < e; ++i) s += a[i];
    int total;
    int run = block_scan_thread(tm, s, scr, &total);
    for (int i = b; i < e; ++i) {
        const int v = a[i];
        a[i] = run;
        run += v;
    }
    tm.sync();
    return total;
}

// The face of a packed row opposite slot s: the other three 16-bit ids,
// ascending, packed into 48 bits.
__device__ __forceinline__ uint64_t face_key(uint2 r, int s) {
    const uint64_t row = uint64_t(r.x) | (uint64_t(r.y) << 32);
    const int sh = 16 * s;
    const uint64_t low = sh ? (row & ((uint64_t(1) << sh) - 1)) : 0ull;
    const uint64_t high = s == 3 ? 0ull : ((row >> (sh + 16)) << sh);
    return low | high;
}

__device__ __forceinline__ uint32_t face_hash(uint64_t key, uint32_t mask) {
    return uint32_t((key * 0x9E3779B97F4A7C15ull) >> 40) & mask;
}

// number of local vertex ids two packed rows have in common
__device__ __forceinline__ int shared_vertices(uint2 a, uint2 b) {
    const uint32_t b0 = b.x & 0xffffu, b1 = b.x >> 16, b2 = b.y & 0xffffu, b3 = b.y >> 16;
    int c = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const uint32_t v = vtx(a, s);
        c += (v == b0) + (v == b1) + (v == b2) + (v == b3);
    }
    return c;
}

// compare-exchange of keys a, b carrying payloads pa, pb
__device__ __forceinline__ void cswap2(int32_t &a, int32_t &b, uint32_t &pa, uint32_t &pb) {
    const bool sw = b < a;
    const int32_t ka = sw ? b : a, kb = sw ? a : b;
    const uint32_t qa = sw ? pb : pa, qb = sw ? pa : pb;
    a = ka;
    b = kb;
    pa = qa;
    pb = qb;
}

// hash entries: bits [0, 20) = 4 * internal-tet index + slot + 1, bits
// [20, 32) = number of other tets matched to the face
constexpr uint32_t kRefMask = (1u << 20) - 1u;
constexpr uint32_t kMatch = 1u << 20;

// ---------------- E'. TT of a non-manifold cluster ----------------
// A triangle of the block lies in three or more tets, so a face may have
// more than one partner.  Every tet of the block holding a face of an
// internal tet is in its TT row, and the block holds them all: such a tet
// holds an own vertex of the face (working set) or lies across a face
// without one (face halo).  Each row is found by comparing vertex triples
// with every tet of the block and sorted by canonical id.  Runs only for
// the clusters the face links mark.  Ends synced.
template <bool COUNT, class Team>
__device__ __forceinline__ void tt_general(const Team &tm, const Smem &S, const uint2 *rows, const int32_t *tmap,
                                        int32_t t_base, int n_ext, int n_own, int n_all, int32_t max_tt,
                                        const WorkItem *it, int64_t *sizes_out, int32_t *err) {
    const int NT = tm.nt(), tid = tm.tid();
    const int n_vtets = n_ext + n_own;
    auto gtet = [&](int loc) -> int32_t {
        if (loc < n_ext) return tmap[loc];
        if (loc < n_vtets) return t_base + (loc - n_ext);
        return tmap[loc - n_own];
    };
    int32_t *tcnt = S.tcnt;
    for (int i = tid; i < n_own; i += NT) {
        const int li = n_ext + i;
        const uint2 r = rows[li];
        int c = 0;
        for (int u = 0; u < n_all; ++u) c += (u != li && shared_vertices(rows[u], r) == 3);
        tcnt[i] = c;
    }
    tm.sync();
    const int tot_tt = block_scan_array(tm, tcnt, n_own, S.scan);
    if (COUNT) {
        if (tid == 0) {
            sizes_out[SZ_TT] = tot_tt;
            sizes_out[SZ_GENERAL] = 1;
        }
    } else {
        if (tot_tt > max_tt) {
            if (tid == 0) atomicOr(err, ERR_CAPACITY);
            tm.sync();
            return;
        }
        for (int i = tid; i < n_own; i += NT) {
            const int li = n_ext + i;
            const uint2 r = rows[li];
            const int p = tcnt[i];
            uint16_t *o = S.st_tt + p;
            int c = 0;
            for (int u = 0; u < n_all; ++u) {
                if (u == li || shared_vertices(rows[u], r) != 3) continue;
                const int32_t gu = gtet(u);
                int q = c++;
                while (q > 0 && gtet(o[q - 1]) > gu) {
                    o[q] = o[q - 1];
                    --q;
                }
                o[q] = uint16_t(u);
            }
            it->tt_off[i] = p;
        }
        if (tid == 0) it->tt_off[n_own] = tot_tt;
        tm.sync();
        copy_out(tm, it->tt_val, tot_tt, [&](int j) { return gtet(S.st_tt[j]); });
    }
    tm.sync();
}

// ---------------------------------------------------------------------------
// One cluster.  COUNT: no output writes; sizes -> sizes_out[5].  SPILL: the
// regions are global scratch and the rows arrive by vector loads instead of
// the bulk copy.  `it` points to a shared-memory copy of the work item; bar
// and phase are the CTA's block-copy barrier and its next parity.  Returns
// false when a bounded wait ran out (the CTA must stop).
// ---------------------------------------------------------------------------
// PART: the item is a part of a cut cluster (block header part != 0); the
// whole-cluster instances carry none of the part logic.
template <bool COUNT, bool SPILL, bool PART, bool GEN, class Team>
__device__ bool run_cluster(const Team &tm, const DevMesh &m, const SmemPlan &plan, const Smem &S, int64_t blk_word, int64_t words,
                            uint32_t mask, const WorkItem *it, int64_t *sizes_out, int32_t *err, uint64_t *bar,
                            uint32_t &phase) {
    const int NT = tm.nt(), NWARP = NT >> 5;
    const int tid = tm.tid(), lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const Caps &caps = plan.caps;
    const int32_t *__restrict__ g = m.blocks + blk_word;
    int32_t *flag = S.scan + 120;  // [0] block fits, [1] bulk copy issued, [2] non-manifold
    const bool jp16 = plan.jpos16 != 0;

    // ---------------- A. the block, by one bulk copy ----------------
    if (tid == 0) {
        const bool fits = words >= kHdrWords && words <= caps.blk_words && (words & 3) == 0;
        int issued = 0;
        if (fits && !SPILL) {
            bulk_load(S.blk, g, uint32_t(4 * words), bar);
            issued = 1;
        }
        flag[0] = fits;
        flag[1] = issued;
        flag[2] = 0;
    }
    tm.sync();
    const bool fits = flag[0] != 0, issued = flag[1] != 0;
    if (!fits) {
        if (tid == 0) atomicOr(err, ERR_CAPACITY);
        tm.sync();
        return true;
    }
    if (SPILL) {
        const int4 *src = reinterpret_cast<const int4 *>(g);
        int4 *dst = reinterpret_cast<int4 *>(S.blk);
        const int n4 = int(words >> 2);
        for (int i = tid; i < n4; i += NT) dst[i] = __ldg(src + i);
        tm.sync();
    } else if (issued) {
        bool ok = mbar_wait(bar, phase);
        if (tm.sync_or(!ok)) {
            if (tid == 0) atomicOr(err, ERR_TIMEOUT);
            if (!ok) mbar_wait(bar, phase);  // the copy may still be in flight
            return false;
        }
        phase ^= 1u;
    }
    const BlockHdr h = *reinterpret_cast<const BlockHdr *>(S.blk);
    // a part block: its record, and the extra tmap words of its internal tets
    const PartInfo *part = (PART && h.part > 0 && h.part <= m.NP) ? m.parts + (h.part - 1) : nullptr;
    const int32_t xmap = part ? h.n_own : 0;
    {
        const int64_t n_tot = int64_t(h.n_ext) + h.n_own + h.n_halo;
        const bool ok = h.n_ext >= 0 && h.n_own >= 0 && h.n_halo >= 0 && h.nv_loc >= 0 && h.own_lo >= 0 &&
                        h.nv_own >= 0 && h.nv_nb >= 0 && h.n_bnd >= 0 && n_tot <= caps.n_tot &&
                        h.n_own <= caps.n_own && h.nv_loc <= caps.nv_loc && h.nv_own <= caps.nv_own &&
                        h.nv_nb <= caps.nv_nb && h.nv_nb <= h.nv_loc && int64_t(h.own_lo) + h.nv_own <= h.nv_nb &&
                        2 * int64_t(h.n_bnd) + 1 <= caps.hcap && (PART ? part != nullptr : h.part == 0) &&
                        blk_words(h.nv_loc, h.n_ext, h.n_own, h.n_halo, h.n_bnd, xmap) == words;
        if (!ok) {
            if (tid == 0) atomicOr(err, ERR_CAPACITY);
            tm.sync();
            return true;
        }
    }
    const int n_ext = h.n_ext, n_own = h.n_own;
    const int n_vtets = n_ext + n_own;
    const uint2 *rows = reinterpret_cast<const uint2 *>(S.blk + blk_rows_off(h.nv_loc, n_ext, h.n_halo, xmap));
    const int32_t *vmap = S.blk + kHdrWords;
    const int32_t *tmap = S.blk + blk_tmap_off(h.nv_loc);
    const int nvo = h.nv_own, lo = h.own_lo;
    const uint32_t nvo_u = uint32_t(nvo);
    // the counting pass sizes the relations the context is preconditioned for
    const bool want_tt = (mask & R_TT) != 0;
    const bool do_vv = !COUNT && (mask & R_VV);
    const bool do_et = !COUNT && (mask & R_ET);
    const int32_t t_base = h.t_base;
    const int n_halo_b = h.n_halo;
    // canonical id of a local tet
    auto gtet = [&](int loc) -> int32_t {
        if (loc < n_ext) return tmap[loc];
        if (loc < n_vtets) return part ? tmap[n_halo_b + loc] : t_base + (loc - n_ext);
        return tmap[loc - n_own];
    };
    // a part writes cluster-level offset values: its entries are shifted by
    // those of the cluster's earlier parts
    int32_t b_vt = 0, b_vv = 0, b_e = 0, b_et = 0;
    if (part && !COUNT) {
        b_vt = __ldg(&part->b_vt);
        b_vv = __ldg(&part->b_vv);
        b_e = __ldg(&part->b_e);
        b_et = __ldg(&part->b_et);
    }

    // The per-own-vertex passes of C2 leave whole warps idle when the cluster
    // has fewer own vertices than the block has threads less a warp: those
    // warps copy VT out meanwhile (vt_off and vt_list do not change after B).
    const int copy_warp0 = (nvo + 31) >> 5;
    const bool vt_copy_later = !COUNT && (mask & R_VT) && copy_warp0 < NWARP &&
                               (COUNT || (mask & (R_VV | R_ET | R_TT)));

    // ---------------- B. VT ----------------
    int vt_total;
    {
        const int pad = plan.pad;
        uint16_t *cw = S.cw;  // [warp][v]: counts, then next position within the row
        uint32_t *cw32 = reinterpret_cast<uint32_t *>(S.cw);
        uint32_t *mk = S.mk;  // [warp][v]: lanes holding v
        const int chunk = ((n_vtets + NWARP - 1) / NWARP + 31) & ~31;
        const int c0 = min(n_vtets, warp * chunk), c1 = min(n_vtets, c0 + chunk);
        fill_words(tm, cw32, (NWARP * pad) >> 1, 0u);  // pad is even
        fill_words(tm, mk, NWARP * pad, 0u);
        tm.sync();
        for (int i = c0 + lane; i < c1; i += 32) {
            const uint2 r = rows[i];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const uint32_t d = vtx(r, s) - uint32_t(lo);
                if (d < nvo_u) atomicAdd(&cw32[(warp * pad + int(d)) >> 1], 1u << (16 * (d & 1u)));
            }
        }
        tm.sync();
        // row lengths -> offsets; every (warp, vertex) gets its first position
        for (int v = tid; v < nvo; v += NT) {
            int tot = 0;
            for (int w = 0; w < NWARP; ++w) tot += int(cw[w * pad + v]);
            S.vt_off[v] = tot;
        }
        tm.sync();
        vt_total = block_scan_array(tm, S.vt_off, nvo, S.scan);
        bool bad = vt_total > caps.n_vt;
        for (int v = tid; v < nvo; v += NT) {
            const int d = (v + 1 < nvo ? S.vt_off[v + 1] : vt_total) - S.vt_off[v];
            bad |= d > caps.max_deg;
            int run = 0;
            for (int w = 0; w < NWARP; ++w) {
                const int c = int(cw[w * pad + v]);
                cw[w * pad + v] = uint16_t(run);
                run += c;
            }
        }
        if (tid == 0) S.vt_off[nvo] = vt_total;
        if (tm.sync_or(bad)) {
            if (tid == 0) atomicOr(err, ERR_CAPACITY);
            return true;
        }
        // fill in tet order, 32 tets per step of each warp; the position
        // of every (tet, own vertex) in that vertex's row is kept for C3/C5
        for (int i0 = c0; i0 < c1; i0 += 32) {
            const int i = i0 + lane;
            const uint2 r = i < c1 ? rows[i] : make_uint2(0xffffffffu, 0xffffffffu);
            uint32_t d[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                d[s] = vtx(r, s) - uint32_t(lo);
                if (d[s] < nvo_u) atomicOr(&mk[warp * pad + d[s]], 1u << lane);
            }
            __syncwarp();
            uint32_t mm[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                mm[s] = 0u;
                if (d[s] < nvo_u) {
                    mm[s] = mk[warp * pad + d[s]];
                    const int pos = int(cw[warp * pad + d[s]]) + __popc(mm[s] & lt);
                    S.vt_list[S.vt_off[d[s]] + pos] = uint16_t(i);
                    if (jp16) reinterpret_cast<uint16_t *>(S.jpos)[4 * i + s] = uint16_t(pos);
                    else S.jpos[4 * i + s] = uint8_t(pos);
                }
            }
            __syncwarp();
#pragma unroll
            for (int s = 0; s < 4; ++s)
                if (d[s] < nvo_u && (mm[s] & lt) == 0u) {
                    cw[warp * pad + d[s]] += uint16_t(__popc(mm[s]));
                    mk[warp * pad + d[s]] = 0u;
                }
            __syncwarp();
        }
        tm.sync();
        if (COUNT) {
            if (tid == 0) sizes_out[SZ_VT] = vt_total;
        } else if ((mask & R_VT) && !vt_copy_later) {
            for (int i = tid; i <= nvo; i += NT) it->vt_off[i] = S.vt_off[i] + b_vt;
            copy_out(tm, it->vt_val, vt_total, [&](int j) { return gtet(S.vt_list[j]); });
        }
    }
    if (!(COUNT || do_vv || do_et || want_tt)) return true;

    // ---------------- C1. neighbour bitmaps, per tet ----------------
    const int W = (h.nv_nb + 31) >> 5;  // bitmap words per vertex
    const int WP = W | 1;                // row stride (odd: rows start in different banks)
    uint32_t *bm = S.bm;
    uint8_t *pre = S.pre;
    fill_words(tm, bm, nvo * WP, 0u);
    if (want_tt) {
        uint32_t *nb32 = reinterpret_cast<uint32_t *>(S.nbr);
        fill_words(tm, nb32, 2 * n_own, FULL);
    }
    tm.sync();
    int etv = 0;  // ET entries: each own vertex of a tet, once per vertex above it
    for (int i = tid; i < n_vtets; i += NT) {
        const uint2 r = rows[i];
        const uint32_t v0 = r.x & 0xffffu, v1 = r.x >> 16, v2 = r.y & 0xffffu, v3 = r.y >> 16;
        uint32_t d = v0 - uint32_t(lo);
        if (d < nvo_u) {
            uint32_t *row = bm + d * WP;
            atomicOr(row + (v1 >> 5), 1u << (v1 & 31));
            atomicOr(row + (v2 >> 5), 1u << (v2 & 31));
            atomicOr(row + (v3 >> 5), 1u << (v3 & 31));
            etv += 3;
        }
        d = v1 - uint32_t(lo);
        if (d < nvo_u) {
            uint32_t *row = bm + d * WP;
            atomicOr(row + (v0 >> 5), 1u << (v0 & 31));
            atomicOr(row + (v2 >> 5), 1u << (v2 & 31));
            atomicOr(row + (v3 >> 5), 1u << (v3 & 31));
            etv += 2;
        }
        d = v2 - uint32_t(lo);
        if (d < nvo_u) {
            uint32_t *row = bm + d * WP;
            atomicOr(row + (v0 >> 5), 1u << (v0 & 31));
            atomicOr(row + (v1 >> 5), 1u << (v1 & 31));
            atomicOr(row + (v3 >> 5), 1u << (v3 & 31));
            etv += 1;
        }
        d = v3 - uint32_t(lo);
        if (d < nvo_u) {
            uint32_t *row = bm + d * WP;
            atomicOr(row + (v0 >> 5), 1u << (v0 & 31));
            atomicOr(row + (v1 >> 5), 1u << (v1 & 31));
            atomicOr(row + (v2 >> 5), 1u << (v2 & 31));
        }
    }
    tm.sync();

    // ---------------- C2. VV rows and owned edges, per own vertex ----------
    int tot[3];  // VV entries, owned edges, ET entries
    {
        // counts per vertex
        for (int x = tid; x < nvo; x += NT) {
            const uint32_t *row = bm + x * WP;
            const int X = lo + x, qx = X >> 5;
            const uint32_t hb = (X & 31) == 31 ? 0u : (FULL << ((X & 31) + 1));
            int cv = 0, ce = 0;
            for (int q = 0; q < W; ++q) {
                const uint32_t w = row[q];
                cv += __popc(w);
                ce += __popc(w & (q < qx ? 0u : (q > qx ? FULL : hb)));
            }
            S.c_vv[x] = cv;
            S.c_e[x] = ce;
        }
        tm.sync();
        // exclusive scans of both count arrays, and the ET total
        {
            const int per = range_len(tm, nvo);
            const int x0 = min(nvo, tid * per), x1 = min(nvo, x0 + per);
            int sv = 0, se = 0;
            for (int x = x0; x < x1; ++x) {
                sv += S.c_vv[x];
                se += S.c_e[x];
            }
            int et0 = etv;
            block_scan3(tm, sv, se, et0, S.scan, tot);
            for (int x = x0; x < x1; ++x) {
                const int a = S.c_vv[x], b = S.c_e[x];
                S.c_vv[x] = sv;
                S.c_e[x] = se;
                sv += a;
                se += b;
            }
            if (tid == 0) {
                S.c_vv[nvo] = tot[0];
                S.c_e[nvo] = tot[1];
            }
        }
        if (tot[1] > caps.max_e || (do_vv && tot[0] > caps.max_vv) || (do_et && tot[2] > caps.max_etv)) {
            if (tid == 0) atomicOr(err, ERR_CAPACITY);
            return true;
        }
        tm.sync();
        if (vt_copy_later && warp >= copy_warp0) {
            // VT out, on the warps the per-vertex loop below leaves idle
            const int t0 = tid - copy_warp0 * 32, nt = NT - copy_warp0 * 32;
            for (int i = t0; i <= nvo; i += nt) it->vt_off[i] = S.vt_off[i] + b_vt;
            int j = t0;
            for (; j + 3 * nt < vt_total; j += 4 * nt) {
                const int32_t a = gtet(S.vt_list[j]), b = gtet(S.vt_list[j + nt]);
                const int32_t c = gtet(S.vt_list[j + 2 * nt]), d = gtet(S.vt_list[j + 3 * nt]);
                it->vt_val[j] = a;
                it->vt_val[j + nt] = b;
                it->vt_val[j + 2 * nt] = c;
                it->vt_val[j + 3 * nt] = d;
            }
            for (; j < vt_total; j += nt) it->vt_val[j] = gtet(S.vt_list[j]);
        }
        // rows: one loop step per set bit, words visited through an
        // occupancy mask; the word holding x keeps its upper bits only and
        // every word with upper bits records the rank of its first one
        bool bad = false;
        for (int x = tid; x < nvo; x += NT) {
            uint32_t *row = bm + x * WP;
            uint8_t *prx = pre + x * WP;
            const int X = lo + x, qx = X >> 5;
            const uint32_t hb = (X & 31) == 31 ? 0u : (FULL << ((X & 31) + 1));
            int vrun = S.c_vv[x], erun = S.c_e[x];
            const int e_first = erun;
            for (int q0 = 0; q0 < W; q0 += 32) {
                const int qn = min(32, W - q0);
                uint32_t occ = 0u;
                for (int u = 0; u < qn; ++u) occ |= (row[q0 + u] != 0u ? 1u : 0u) << u;
                uint32_t w = 0u, um = 0u;
                int q = 0;
                for (;;) {
                    if (w == 0u) {
                        if (occ == 0u) break;
                        q = q0 + __ffs(occ) - 1;
                        occ &= occ - 1u;
                        w = row[q];
                        um = q < qx ? 0u : (q > qx ? FULL : hb);
                        if (w & um) prx[q] = uint8_t(erun - e_first);
                        if (q == qx) row[q] = w & hb;
                    }
                    const uint32_t bit = w & (0u - w);
                    w ^= bit;
                    const uint16_t id = uint16_t(q * 32 + __ffs(bit) - 1);
                    if (do_vv) S.st_v[vrun] = id;
                    ++vrun;
                    if (bit & um) {
                        if (do_et) S.st_w[erun] = id;
                        ++erun;
                    }
                }
            }
            bad |= erun - e_first > 255;
        }
        if (tm.sync_or(bad)) {
            if (tid == 0) atomicOr(err, ERR_CAPACITY);
            return true;
        }
        if (COUNT && tid == 0) {
            sizes_out[SZ_VV] = tot[0];
            sizes_out[SZ_E] = tot[1];
            sizes_out[SZ_ET] = tot[2];
        }
        if (do_vv) {
            for (int i = tid; i <= nvo; i += NT) it->vv_off[i] = S.c_vv[i] + b_vv;
            copy_out(tm, it->vv_val, tot[0], [&](int j) { return vmap[S.st_v[j]]; });
        }
        if (do_et) {
            for (int i = tid; i <= nvo; i += NT) it->eu_off[i] = S.c_e[i] + b_e;
            copy_out(tm, it->e_w, tot[1], [&](int e) { return vmap[S.st_w[e]]; });
            if (tid == 0) it->et_off[tot[1]] = tot[2] + b_et;
        }
    }
    if (!(do_et || want_tt)) return true;
    const int tot_e = tot[1], tot_etv = tot[2];
    const int nch = plan.nch;
    uint32_t *em = S.emask;
    tm.sync();  // VV and endpoint staging are dead: r2 takes the edge masks
    fill_words(tm, em, tot_e * nch, 0u);
    tm.sync();

    // ---------------- C3. edge tet masks, per tet ----------------
    // bit j of mask(x, w): the j-th tet of VT(x) contains w; every own
    // vertex x of a tet marks the edges to the tet's vertices above x
    {
        auto mark = [&](uint32_t x, uint32_t y, uint32_t j) {
            const int q = int(y >> 5);
            const int e = S.c_e[x] + int(pre[x * WP + q]) + __popc(bm[x * WP + q] & ((1u << (y & 31)) - 1u));
            atomicOr(em + e * nch + (j >> 5), 1u << (j & 31));
        };
        for (int i = tid; i < n_vtets; i += NT) {
            const uint2 r = rows[i];
            const uint32_t v0 = r.x & 0xffffu, v1 = r.x >> 16, v2 = r.y & 0xffffu, v3 = r.y >> 16;
            uint32_t j0, j1, j2;
            if (jp16) {
                const uint2 jw = reinterpret_cast<const uint2 *>(S.jpos)[i];
                j0 = jw.x & 0xffffu;
                j1 = jw.x >> 16;
                j2 = jw.y & 0xffffu;
            } else {
                const uint32_t jw = reinterpret_cast<const uint32_t *>(S.jpos)[i];
                j0 = jw & 0xffu;
                j1 = (jw >> 8) & 0xffu;
                j2 = (jw >> 16) & 0xffu;
            }
            const uint32_t x0 = v0 - uint32_t(lo), x1 = v1 - uint32_t(lo), x2 = v2 - uint32_t(lo);
            if (x0 < nvo_u) {
                mark(x0, v1, j0);
                mark(x0, v2, j0);
                mark(x0, v3, j0);
            }
            if (x1 < nvo_u) {
                mark(x1, v2, j1);
                mark(x1, v3, j1);
            }
            if (x2 < nvo_u) mark(x2, v3, j2);
        }
    }
    tm.sync();

    // ---------------- C5. TT links of faces with an own lowest vertex ------
    if (want_tt) {
        int32_t flags = 0;
        for (int i = tid; i < n_own; i += NT) {
            const int li = n_ext + i;
            const uint2 r = rows[li];
            const uint32_t v0 = r.x & 0xffffu, v1 = r.x >> 16, v2 = r.y & 0xffffu, v3 = r.y >> 16;
            const uint32_t a = v0 - uint32_t(lo);
            if (a >= nvo_u) {  // an internal tet's lowest vertex is own (a part's: an earlier part's)
                if (!part) flags |= ERR_BAD_BLOCK;
                continue;
            }
            auto rank = [&](uint32_t x, uint32_t y) -> int {
                const int q = int(y >> 5);
                return S.c_e[x] + int(pre[x * WP + q]) + __popc(bm[x * WP + q] & ((1u << (y & 31)) - 1u));
            };
            // partner of tet li across the face (x, w1, w2): the set bit of
            // mask(x, w1) & mask(x, w2) other than li's own position js in VT(x)
            auto link = [&](int e1, int e2, int base, int js, int opp) {
                const int cs = js >> 5;
                const uint32_t sb = 1u << (js & 31);
                int found = 0, partner = -1;
                for (int c = 0; c < nch; ++c) {
                    uint32_t mm = em[e1 * nch + c] & em[e2 * nch + c];
                    if (c == cs) mm &= ~sb;
                    found += __popc(mm);
                    if (mm != 0u && partner < 0) partner = S.vt_list[base + c * 32 + __ffs(mm) - 1];
                }
                if (found > 1) flags |= ERR_NONMANIFOLD;
                if (partner >= 0) S.nbr[i * 4 + opp] = uint16_t(partner);
            };
            const int e1 = rank(a, v1), e2 = rank(a, v2), e3 = rank(a, v3);
            const int ja = jp16 ? reinterpret_cast<const uint16_t *>(S.jpos)[4 * li] : S.jpos[4 * li];
            const int jb = jp16 ? reinterpret_cast<const uint16_t *>(S.jpos)[4 * li + 1] : S.jpos[4 * li + 1];
            const int base_a = S.vt_off[a];
            link(e1, e2, base_a, ja, 3);
            link(e1, e3, base_a, ja, 2);
            link(e2, e3, base_a, ja, 1);
            const uint32_t b = v1 - uint32_t(lo);
            if (b < nvo_u) link(rank(b, v2), rank(b, v3), S.vt_off[b], jb, 0);
        }
        if (GEN && !PART && (flags & ERR_NONMANIFOLD)) {  // TT of this cluster takes the general pass (E')
            flag[2] = 1;
            flags &= ~ERR_NONMANIFOLD;
        }
        if (flags) atomicOr(err, flags);
    }
    tm.sync();  // bitmaps and rank prefixes are dead: r1 takes the ET staging

    // ---------------- C4. ET rows, per edge ----------------
    if (do_et) {
        uint16_t *st_et = S.st_et;
        const int per = range_len(tm, tot_e);
        const int e0 = min(tot_e, tid * per), e1 = min(tot_e, e0 + per);
        int cnt = 0;
        for (int e = e0; e < e1; ++e)
            for (int c = 0; c < nch; ++c) cnt += __popc(em[e * nch + c]);
        int total;
        int run = block_scan_thread(tm, cnt, S.scan, &total);
        if (total != tot_etv) {  // every (own vertex, tet, upper vertex) sets one distinct bit
            if (tid == 0) atomicOr(err, ERR_BAD_BLOCK);
            tm.sync();
            return true;
        }
        // own vertex holding edge e0: the largest x with c_e[x] <= e0
        int xe = 0;
        if (e0 < e1) {
            int hi = nvo - 1;
            while (xe < hi) {
                const int mid = (xe + hi + 1) >> 1;
                if (S.c_e[mid] <= e0) xe = mid;
                else hi = mid - 1;
            }
        }
        for (int e = e0; e < e1; ++e) {
            while (S.c_e[xe + 1] <= e) ++xe;
            const int base = S.vt_off[xe];
            const int t0 = run;
            for (int c = 0; c < nch; ++c) {
                uint32_t mm = em[e * nch + c];
                while (mm) {
                    const int b = __ffs(mm) - 1;
                    mm &= mm - 1;
                    st_et[run++] = S.vt_list[base + c * 32 + b];
                }
            }
            em[e * nch] = uint32_t(t0);  // the edge's first mask word now holds its row offset
        }
        tm.sync();
        for (int e = tid; e < tot_e; e += NT) it->et_off[e] = int32_t(em[e * nch]) + b_et;
        copy_out(tm, it->et_val, tot_etv, [&](int j) { return gtet(st_et[j]); });
        tm.sync();  // ET staging is dead: r1 takes the face hash
    }

    if (want_tt) {
        // ---------------- D. faces with no own vertex, against the halo ----
        const uint32_t hmask = uint32_t(caps.hcap - 1);
        uint32_t *hash = S.hash;
        fill_words(tm, hash, caps.hcap, 0u);
        tm.sync();
        int32_t flags = 0;
        // the internal tets whose face (b, c, d) has no own vertex
        const uint16_t *bnd =
            reinterpret_cast<const uint16_t *>(S.blk + blk_bnd_off(h.nv_loc, n_ext, n_own, h.n_halo, xmap));
        for (int jb = tid; jb < h.n_bnd; jb += NT) {
            const int i = bnd[jb];
            const uint2 r = rows[n_ext + i];
            const uint64_t key = face_key(r, 0);
            uint32_t hp = face_hash(key, hmask);
            int probe = 0;
            for (; probe < caps.hcap; ++probe) {
                const uint32_t prev = atomicCAS(&hash[hp], 0u, uint32_t(i * 4 + 1));
                if (prev == 0u) break;
                const uint32_t ref = (prev & kRefMask) - 1u;
                if (face_key(rows[n_ext + (ref >> 2)], 0) == key) {
                    if (atomicAdd(&hash[hp], kMatch) >= kMatch) flags |= ERR_NONMANIFOLD;
                    S.nbr[ref] = uint16_t(n_ext + i);
                    S.nbr[i * 4] = uint16_t(n_ext + (ref >> 2));
                    break;
                }
                hp = (hp + 1u) & hmask;
            }
            if (probe == caps.hcap) flags |= ERR_HASH_FULL;
        }
        tm.sync();
        const int n_halo = h.n_halo;
        for (int j = tid; j < 4 * n_halo; j += NT) {  // one (halo tet, face) per step
            const int tl = n_vtets + (j >> 2);
            const uint64_t key = face_key(rows[tl], j & 3);
            uint32_t hp = face_hash(key, hmask);
            for (int probe = 0; probe < caps.hcap; ++probe) {
                const uint32_t e = hash[hp];
                if (e == 0u) break;
                const uint32_t ref = (e & kRefMask) - 1u;
                if (face_key(rows[n_ext + (ref >> 2)], 0) == key) {
                    if (atomicAdd(&hash[hp], kMatch) >= kMatch) flags |= ERR_NONMANIFOLD;
                    S.nbr[ref] = uint16_t(tl);
                    break;
                }
                hp = (hp + 1u) & hmask;
            }
        }
        if (GEN && !PART && (flags & ERR_NONMANIFOLD)) {
            flag[2] = 1;
            flags &= ~ERR_NONMANIFOLD;
        }
        if (flags) atomicOr(err, flags);
        tm.sync();
        if (GEN && !PART && flag[2] != 0) {
            tt_general<COUNT>(tm, S, rows, tmap, t_base, n_ext, n_own, n_vtets + h.n_halo, caps.max_tt, it,
                              sizes_out, err);
            return true;
        }
        // ---------------- E. TT rows ----------------
        int32_t *tcnt = S.tcnt;
        for (int i = tid; i < n_own; i += NT) {
            const uint2 nb = *reinterpret_cast<const uint2 *>(&S.nbr[i * 4]);
            tcnt[i] = ((nb.x & 0xffffu) != 0xffffu) + ((nb.x >> 16) != 0xffffu) + ((nb.y & 0xffffu) != 0xffffu) +
                      ((nb.y >> 16) != 0xffffu);
        }
        tm.sync();
        if (COUNT && part) {
            // row lengths of the part's own internal tets, by canonical id
            for (int i = tid; i < n_own; i += NT)
                if ((rows[n_ext + i].x & 0xffffu) - uint32_t(lo) < nvo_u) m.tt_pos[gtet(n_ext + i)] = tcnt[i];
            tm.sync();
        }
        const int tot_tt = block_scan_array(tm, tcnt, n_own, S.scan);
        if (COUNT) {
            if (tid == 0) sizes_out[SZ_TT] = tot_tt;
        } else if (part) {
            // rows straight to their cluster-level offsets (the earlier parts'
            // rows of the same cluster precede this part's in the list)
            if (tot_tt > caps.max_tt) {
                if (tid == 0) atomicOr(err, ERR_CAPACITY);
                return true;
            }
            int32_t *const c_off = it->tt_off - __ldg(&part->b_to);
            int32_t *const c_val = it->tt_val - __ldg(&part->b_tt);
            const int32_t tb = __ldg(&part->t_base_c);
            for (int i = tid; i < n_own; i += NT) {
                if ((rows[n_ext + i].x & 0xffffu) - uint32_t(lo) >= nvo_u) continue;  // an earlier part's row
                const uint2 nb = *reinterpret_cast<const uint2 *>(&S.nbr[i * 4]);
                const uint32_t n0 = nb.x & 0xffffu, n1 = nb.x >> 16, n2 = nb.y & 0xffffu, n3 = nb.y >> 16;
                int32_t w0 = n0 != 0xffffu ? gtet(int32_t(n0)) : INT32_MAX;
                int32_t w1 = n1 != 0xffffu ? gtet(int32_t(n1)) : INT32_MAX;
                int32_t w2 = n2 != 0xffffu ? gtet(int32_t(n2)) : INT32_MAX;
                int32_t w3 = n3 != 0xffffu ? gtet(int32_t(n3)) : INT32_MAX;
                uint32_t l0 = n0, l1 = n1, l2 = n2, l3 = n3;
                cswap2(w0, w1, l0, l1); cswap2(w2, w3, l2, l3); cswap2(w0, w2, l0, l2); cswap2(w1, w3, l1, l3);
                cswap2(w1, w2, l1, l2);
                const int32_t gt = gtet(n_ext + i);
                const int32_t p = m.tt_pos[gt];
                c_off[gt - tb] = p;
                if (w0 != INT32_MAX) c_val[p] = w0;
                if (w1 != INT32_MAX) c_val[p + 1] = w1;
                if (w2 != INT32_MAX) c_val[p + 2] = w2;
                if (w3 != INT32_MAX) c_val[p + 3] = w3;
            }
            if (tid == 0 && __ldg(&part->last)) c_off[__ldg(&part->n_own_c)] = __ldg(&part->tt_total);
        } else {
            if (tot_tt > caps.max_tt) {
                if (tid == 0) atomicOr(err, ERR_CAPACITY);
                return true;
            }
            for (int i = tid; i < n_own; i += NT) {
                const uint2 nb = *reinterpret_cast<const uint2 *>(&S.nbr[i * 4]);
                const uint32_t n0 = nb.x & 0xffffu, n1 = nb.x >> 16, n2 = nb.y & 0xffffu, n3 = nb.y >> 16;
                // local ids ordered by canonical id; absent neighbours sort last
                int32_t w0 = n0 != 0xffffu ? gtet(int32_t(n0)) : INT32_MAX;
                int32_t w1 = n1 != 0xffffu ? gtet(int32_t(n1)) : INT32_MAX;
                int32_t w2 = n2 != 0xffffu ? gtet(int32_t(n2)) : INT32_MAX;
                int32_t w3 = n3 != 0xffffu ? gtet(int32_t(n3)) : INT32_MAX;
                uint32_t l0 = n0, l1 = n1, l2 = n2, l3 = n3;
                cswap2(w0, w1, l0, l1); cswap2(w2, w3, l2, l3); cswap2(w0, w2, l0, l2); cswap2(w1, w3, l1, l3);
                cswap2(w1, w2, l1, l2);
                // canonical ids straight out: a warp's rows are adjacent, so
                // its four stores cover one contiguous span
                const int p = tcnt[i];
                it->tt_off[i] = p;
                int32_t *o = it->tt_val + p;
                if (w0 != INT32_MAX) o[0] = w0;
                if (w1 != INT32_MAX) o[1] = w1;
                if (w2 != INT32_MAX) o[2] = w2;
                if (w3 != INT32_MAX) o[3] = w3;
            }
            if (tid == 0) it->tt_off[n_own] = tot_tt;
        }
    }
    tm.sync();
    return true;
}

// A work item: a whole cluster, or (id >= K) a part of a cut cluster.  GEN:
// the whole-cluster instance carries the general TT pass (E'); the hot
// shared-memory kernel leaves it out, and the clusters that need it (the
// counting pass marks them) run from per-item bins.
template <bool COUNT, bool SPILL, bool GEN>
__device__ __forceinline__ bool run_item(bool part, const DevMesh &m, const SmemPlan &plan, const Smem &S,
                                         int64_t blk_word, int64_t words, uint32_t mask, const WorkItem *it,
                                         int64_t *sizes_out, int32_t *err, uint64_t *bar, uint32_t &phase) {
    const BlockTeam tm;
    if (part)
        return run_cluster<COUNT, SPILL, true, false>(tm, m, plan, S, blk_word, words, mask, it, sizes_out, err, bar,
                                                      phase);
    return run_cluster<COUNT, SPILL, false, GEN>(tm, m, plan, S, blk_word, words, mask, it, sizes_out, err, bar, phase);
}

// SPILL: the cluster's regions live in a per-CTA slice of global scratch
// (clusters whose working set exceeds shared memory); otherwise in dynamic
// shared memory.
template <bool SPILL>
__device__ __forceinline__ char *region_base(char *smem, char *gscratch, const SmemPlan &plan) {
    return SPILL ? gscratch + size_t(blockIdx.x) * size_t(plan.total) : smem;
}

// Blocks have up to 1024 threads, so every cluster kernel is bounded to 64
// registers per thread.
constexpr int kMaxThreads = 1024;

template <bool SPILL>
__device__ __forceinline__ void init_barrier(uint64_t *bar) {
    if (!SPILL && threadIdx.x == 0) mbar_init(bar);
    __syncthreads();
}

template <bool SPILL>
__global__ void __launch_bounds__(kMaxThreads) count_kernel(DevMesh m, SmemPlan plan, const int32_t *ids, int32_t n, int64_t *sizes, int32_t *err,
                             int32_t *ticket, char *gscratch, uint32_t mask) {
    extern __shared__ __align__(16) char smem[];
    const Smem S = carve(region_base<SPILL>(smem, gscratch, plan), plan);
    __shared__ int32_t s_idx;
    __shared__ int64_t s_sizes[SZ_N + 1];
    __shared__ __align__(8) uint64_t s_bar;
    init_barrier<SPILL>(&s_bar);
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(ticket, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= n) break;
        const int k = ids ? ids[idx] : idx;
        if (k < 0 || k >= m.K + m.NP) {
            if (threadIdx.x == 0) atomicOr(err, ERR_BAD_ITEM);
            continue;
        }
        if (threadIdx.x <= SZ_N) s_sizes[threadIdx.x] = 0;
        __syncthreads();
        if (!run_item<true, SPILL, true>(k >= m.K, m, plan, S, m.blk_off[k], m.blk_off[k + 1] - m.blk_off[k], mask, nullptr, s_sizes,
                                      err, &s_bar, phase))
            return;
        __syncthreads();
        if (threadIdx.x < SZ_N) sizes[int64_t(k) * SZ_N + threadIdx.x] = s_sizes[threadIdx.x];
        if (threadIdx.x == 0 && k < m.K && m.tt_general) m.tt_general[k] = int32_t(s_sizes[SZ_GENERAL]);
    }
}

template <bool SPILL>
__global__ void __launch_bounds__(kMaxThreads) build_kernel(DevMesh m, SmemPlan plan, const WorkItem *items, const int32_t *order, int32_t n,
                             int32_t *err, int32_t *ticket, char *gscratch) {
    extern __shared__ __align__(16) char smem[];
    const Smem S = carve(region_base<SPILL>(smem, gscratch, plan), plan);
    __shared__ int32_t s_idx;
    __shared__ WorkItem s_item;
    __shared__ __align__(8) uint64_t s_bar;
    init_barrier<SPILL>(&s_bar);
    uint32_t phase = 0;
    if (threadIdx.x == 0) s_idx = atomicAdd(ticket, 1);
    for (;;) {
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= n) break;
        if (threadIdx.x == 0) {
            s_item = items[order ? order[idx] : idx];
            s_idx = atomicAdd(ticket, 1);  // the next cluster of this CTA
        }
        __syncthreads();
        if (threadIdx.x == 32 && s_idx < n) {
            // its block into L2 while this cluster builds
            const int k2 = items[order ? order[s_idx] : s_idx].k;
            if (k2 >= 0 && k2 < m.K + m.NP) {
                const int64_t w0 = m.blk_off[k2], w1 = m.blk_off[k2 + 1];
                if (w1 > w0) prefetch_l2(m.blocks + w0, uint32_t(4 * (w1 - w0)));
            }
        }
        const int k = s_item.k;
        if (k < 0 || k >= m.K + m.NP) {
            if (threadIdx.x == 0) atomicOr(err, ERR_BAD_ITEM);
            continue;
        }
        if (!run_item<false, SPILL, SPILL>(k >= m.K, m, plan, S, s_item.blk, m.blk_off[k + 1] - m.blk_off[k], s_item.mask, &s_item,
                                       nullptr, err, &s_bar, phase))
            return;
    }
}

template <bool SPILL>
__global__ void __launch_bounds__(kMaxThreads) build_one_kernel(DevMesh m, SmemPlan plan, const WorkItem *items, int32_t index, int32_t *err,
                                 char *gscratch) {
    extern __shared__ __align__(16) char smem[];
    const Smem S = carve(region_base<SPILL>(smem, gscratch, plan), plan);
    __shared__ WorkItem s_item;
    __shared__ __align__(8) uint64_t s_bar;
    init_barrier<SPILL>(&s_bar);
    uint32_t phase = 0;
    if (threadIdx.x == 0) s_item = items[index];
    __syncthreads();
    if (s_item.k < 0 || s_item.k >= m.K + m.NP) {
        if (threadIdx.x == 0) atomicOr(err, ERR_BAD_ITEM);
        return;
    }
    run_cluster<false, SPILL, false, true>(BlockTeam{}, m, plan, S, s_item.blk, m.blk_off[s_item.k + 1] - m.blk_off[s_item.k], s_item.mask,
                              &s_item, nullptr, err, &s_bar, phase);
}

// ---------------------------------------------------------------------------
// Several small clusters per CTA.  Each team of team_n threads (a multiple
// of 32; the block holds blockDim.x / team_n teams) takes clusters from the
// ticket on its own and builds each in its own slice of the dynamic shared
// memory, with a named barrier and a bulk-copy barrier of its own, so a
// small cluster's barriers involve only its team.
// ---------------------------------------------------------------------------
constexpr int kMaxTeams = 15;  // named barriers 1..15
constexpr int kMaxTeamBlock = 512;

__global__ void __launch_bounds__(kMaxTeamBlock) build_kernel_team(DevMesh m, SmemPlan plan, const WorkItem *items,
                                                                const int32_t *order, int32_t n, int32_t *err,
                                                                int32_t *ticket, int team_n) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int32_t s_idx[kMaxTeams];
    __shared__ WorkItem s_item[kMaxTeams];
    __shared__ __align__(8) uint64_t s_bar[kMaxTeams];
    const int g = int(threadIdx.x) / team_n;
    if (g >= kMaxTeams) return;  // (the host never launches more teams)
    const SliceTeam tm{team_n, int(threadIdx.x) - g * team_n, 1 + g};
    const Smem S = carve(smem + size_t(g) * size_t(plan.total), plan);
    if (tm.tid() == 0) mbar_init(&s_bar[g]);
    tm.sync();
    uint32_t phase = 0;
    for (;;) {
        if (tm.tid() == 0) {
            const int idx = atomicAdd(ticket, 1);
            s_idx[g] = idx;
            if (idx < n) s_item[g] = items[order ? order[idx] : idx];
        }
        tm.sync();
        if (s_idx[g] >= n) break;
        const int k = s_item[g].k;
        if (k < 0 || k >= m.K) {
            if (tm.tid() == 0) atomicOr(err, ERR_BAD_ITEM);
            tm.sync();
            continue;
        }
        if (!run_cluster<false, false, false, false>(tm, m, plan, S, s_item[g].blk, m.blk_off[k + 1] - m.blk_off[k],
                                              s_item[g].mask, &s_item[g], nullptr, err, &s_bar[g], phase))
            return;
        tm.sync();  // the next claim rewrites this team's item
    }
}

// ---------------------------------------------------------------------------
// Clusters that each carry their own shared-memory plan (plans[k]), for the
// largest clusters, whose plans cannot be merged under one launch plan
// without exceeding a CTA's shared memory: every CTA copies its cluster's
// plan into shared memory and carves its regions from it, so such clusters
// of uneven sizes still share one persistent launch, with the dynamic shared
// memory of the largest.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_plan(SmemPlan &dst, const SmemPlan *src) {
    constexpr int kWords = int(sizeof(SmemPlan) / 4);
    for (int i = threadIdx.x; i < kWords; i += blockDim.x)
        reinterpret_cast<int32_t *>(&dst)[i] = reinterpret_cast<const int32_t *>(src)[i];
}

__global__ void __launch_bounds__(kMaxThreads) count_kernel_pi(DevMesh m, const SmemPlan *plans, const int32_t *ids,
                                                              int32_t n, int64_t *sizes, int32_t *err, int32_t *ticket,
                                                              uint32_t mask) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int32_t s_idx;
    __shared__ int64_t s_sizes[SZ_N + 1];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ __align__(16) SmemPlan s_plan;
    init_barrier<false>(&s_bar);
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(ticket, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= n) break;
        const int k = ids ? ids[idx] : idx;
        if (k < 0 || k >= m.K + m.NP) {
            if (threadIdx.x == 0) atomicOr(err, ERR_BAD_ITEM);
            continue;
        }
        load_plan(s_plan, plans + k);
        if (threadIdx.x <= SZ_N) s_sizes[threadIdx.x] = 0;
        __syncthreads();
        const Smem S = carve(smem, s_plan);
        if (!run_item<true, false, true>(k >= m.K, m, s_plan, S, m.blk_off[k], m.blk_off[k + 1] - m.blk_off[k], mask, nullptr,
                                      s_sizes, err, &s_bar, phase))
            return;
        __syncthreads();
        if (threadIdx.x < SZ_N) sizes[int64_t(k) * SZ_N + threadIdx.x] = s_sizes[threadIdx.x];
        if (threadIdx.x == 0 && k < m.K && m.tt_general) m.tt_general[k] = int32_t(s_sizes[SZ_GENERAL]);
    }
}

__global__ void __launch_bounds__(kMaxThreads) build_kernel_pi(DevMesh m, const SmemPlan *plans, const WorkItem *items,
                                                              const int32_t *order, int32_t n, int32_t *err,
                                                              int32_t *ticket) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int32_t s_idx;
    __shared__ WorkItem s_item;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ __align__(16) SmemPlan s_plan;
    init_barrier<false>(&s_bar);
    uint32_t phase = 0;
    if (threadIdx.x == 0) s_idx = atomicAdd(ticket, 1);
    for (;;) {
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= n) break;
        if (threadIdx.x == 0) {
            s_item = items[order ? order[idx] : idx];
            s_idx = atomicAdd(ticket, 1);  // the next cluster of this CTA
        }
        __syncthreads();
        if (threadIdx.x == 32 && s_idx < n) {
            const int k2 = items[order ? order[s_idx] : s_idx].k;
            if (k2 >= 0 && k2 < m.K + m.NP) {
                const int64_t w0 = m.blk_off[k2], w1 = m.blk_off[k2 + 1];
                if (w1 > w0) prefetch_l2(m.blocks + w0, uint32_t(4 * (w1 - w0)));
            }
        }
        const int k = s_item.k;
        if (k < 0 || k >= m.K + m.NP) {
            if (threadIdx.x == 0) atomicOr(err, ERR_BAD_ITEM);
            continue;
        }
        load_plan(s_plan, plans + k);
        __syncthreads();
        const Smem S = carve(smem, s_plan);
        if (!run_item<false, false, true>(k >= m.K, m, s_plan, S, s_item.blk, m.blk_off[k + 1] - m.blk_off[k], s_item.mask, &s_item,
                                       nullptr, err, &s_bar, phase))
            return;
    }
}

// ---------------------------------------------------------------------------
// Device-resident serving loop.  Work items arrive in a ring in mapped host
// memory; the host writes an item and then publishes its ticket by a release
// store of the ring tail.  Each CTA claims the next published ticket (acquire
// load of the tail at system scope, CAS on a device counter), builds the
// cluster into the cache slot the item points to, then fences and stores the
// ticket into the slot's done flag (release, system scope).  A CTA that finds
// no published work sleeps and polls again; after idle_ns without a claim,
// or when the host raises the stop flag, it returns.  Every wait is bounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long ld_acquire_sys(const long long *p) {
    long long v;
    asm volatile("ld.acquire.sys.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_sys32(const int *p) {
    int v;
    asm volatile("ld.acquire.sys.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(long long *p, long long v) {
    asm volatile("st.release.sys.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(1024) serve_kernel(DevMesh m, const SmemPlan *plans, ServeRing ring,
                                                     int32_t *err) {
    extern __shared__ __align__(16) char smem[];
    __shared__ __align__(16) SmemPlan s_plan;
    __shared__ long long s_t;
    __shared__ WorkItem s_item;
    __shared__ __align__(8) uint64_t s_bar;
    init_barrier<false>(&s_bar);
    uint32_t phase = 0;
    unsigned long long last = globaltimer();
    __shared__ unsigned long long s_claim;
    for (;;) {
        if (threadIdx.x == 0) {
            long long t = -1;
            unsigned sleep_ns = 256;
            for (;;) {
                if (ld_acquire_sys32(ring.stop)) break;
                const long long pub = ld_acquire_sys(ring.tail);
                const unsigned long long cur = *reinterpret_cast<volatile unsigned long long *>(ring.next);
                if ((long long)cur < pub) {
                    if (atomicCAS(ring.next, cur, cur + 1ull) == cur) {
                        t = (long long)cur;
                        break;
                    }
                    continue;
                }
                if (globaltimer() - last > ring.idle_ns) break;
                __nanosleep(sleep_ns);
                if (sleep_ns < 2048) sleep_ns *= 2;
            }
            if (t >= 0) {
                s_claim = globaltimer();
                const int slot = int(t % ring.cap);
                const volatile int32_t *src = reinterpret_cast<const volatile int32_t *>(ring.items + slot);
                int32_t *dst = reinterpret_cast<int32_t *>(&s_item);
                for (int w = 0; w < int(sizeof(WorkItem) / 4); ++w) dst[w] = src[w];
            }
            s_t = t;
        }
        __syncthreads();
        const long long t = s_t;
        if (t < 0) break;
        bool go_on = true;
        if (s_item.k >= 0 && s_item.k < m.K) {
            load_plan(s_plan, plans + s_item.k);  // the cluster's own plan
            __syncthreads();
            const Smem S = carve(smem, s_plan);
            go_on = run_cluster<false, false, false, true>(BlockTeam{}, m, s_plan, S, s_item.blk, m.blk_off[s_item.k + 1] - m.blk_off[s_item.k],
                                              s_item.mask, &s_item, nullptr, err, &s_bar, phase);
        } else if (threadIdx.x == 0) {
            atomicOr(err, ERR_BAD_ITEM);
        }
        if (!go_on) break;  // a bounded wait ran out; the slot stays not done
        __syncthreads();
        if (threadIdx.x == 0) {
            const int slot = int(t % ring.cap);
            ring.times[2 * slot] = (long long)s_claim;
            ring.times[2 * slot + 1] = (long long)globaltimer();
            __threadfence_system();
            st_release_sys(ring.done + slot, t);
        }
        last = globaltimer();
    }
}

// Output placement: exclusive scans, over the listed clusters, of the
// lengths of the ten output arrays, then one work item per cluster with its
// output pointers.  Three launches: block sums, a scan of the block sums,
// then per-block scans that write the items.  arrays_base holds the base
// pointers of the ten output arrays (its k / mask / blk fields are ignored).
constexpr int kBasesThreads = 256;
constexpr int NA = 10;

__device__ __forceinline__ void item_lengths(const DevMesh &m, const int32_t *ids, const int64_t *sizes,
                                             uint32_t mask, int idx, int64_t *L) {
    const int k = ids ? ids[idx] : idx;
    const int64_t *sz = sizes + int64_t(k) * SZ_N;
    // a cluster's offset arrays end with one extra entry; a part's only when
    // it is its cluster's last
    int64_t nvo, nown, fin;
    if (k < m.K) {
        nvo = m.I_V[k + 1] - m.I_V[k];
        nown = m.I_T[k + 1] - m.I_T[k];
        fin = 1;
    } else {
        const PartInfo &p = m.parts[k - m.K];
        nvo = p.nvo;
        nown = p.n_rows;
        fin = p.last;
    }
    const bool vt = mask & R_VT, vv = mask & R_VV, et = mask & R_ET, tt = mask & R_TT;
    L[0] = vt ? nvo + fin : 0;
    L[1] = vt ? sz[SZ_VT] : 0;
    L[2] = vv ? nvo + fin : 0;
    L[3] = vv ? sz[SZ_VV] : 0;
    L[4] = et ? nvo + fin : 0;
    L[5] = et ? sz[SZ_E] : 0;
    L[6] = et ? sz[SZ_E] + fin : 0;
    L[7] = et ? sz[SZ_ET] : 0;
    L[8] = tt ? nown + fin : 0;
    L[9] = tt ? sz[SZ_TT] : 0;
}

// block-wide exclusive scan of NA int64 values per thread; totals -> tot[]
__device__ __forceinline__ void block_scan_na(int64_t *v, int64_t (*s_warp)[NA], int64_t *tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t incl[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        int64_t x = v[a];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        incl[a] = x;
        if (lane == 31) s_warp[warp][a] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int64_t w = lane < nw ? s_warp[lane][a] : 0;
            int64_t x = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += y;
            }
            if (lane < nw) s_warp[lane][a] = x - w;
            if (lane == 31) tot[a] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < NA; ++a) v[a] = s_warp[warp][a] + incl[a] - v[a];
}

__global__ void __launch_bounds__(kBasesThreads) bases_sum_kernel(DevMesh m, const int32_t *ids, int32_t n,
                                                                  const int64_t *sizes, uint32_t mask,
                                                                  int64_t *bsum) {
    __shared__ int64_t s_warp[32][NA];
    __shared__ int64_t s_tot[NA];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int64_t L[NA];
    if (idx < n) item_lengths(m, ids, sizes, mask, idx, L);
    else
        for (int a = 0; a < NA; ++a) L[a] = 0;
    block_scan_na(L, s_warp, s_tot);
    if (threadIdx.x < NA) bsum[int64_t(blockIdx.x) * NA + threadIdx.x] = s_tot[threadIdx.x];
}

__global__ void __launch_bounds__(kBasesThreads) bases_scan_kernel(int32_t nblocks, int64_t *bsum,
                                                                   int64_t *totals) {
    __shared__ int64_t s_warp[32][NA];
    __shared__ int64_t s_tot[NA];
    __shared__ int64_t s_run[NA];
    if (threadIdx.x < NA) s_run[threadIdx.x] = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblocks; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        int64_t v[NA];
        for (int a = 0; a < NA; ++a) v[a] = b < nblocks ? bsum[int64_t(b) * NA + a] : 0;
        block_scan_na(v, s_warp, s_tot);
        if (b < nblocks)
            for (int a = 0; a < NA; ++a) bsum[int64_t(b) * NA + a] = v[a] + s_run[a];
        __syncthreads();
        if (threadIdx.x < NA) s_run[threadIdx.x] += s_tot[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x < NA) totals[threadIdx.x] = s_run[threadIdx.x];
}

__global__ void __launch_bounds__(kBasesThreads) bases_write_kernel(DevMesh m, const int32_t *ids, int32_t n,
                                                                    const int64_t *sizes, uint32_t mask,
                                                                    const WorkItem *arrays_base,
                                                                    const int64_t *bsum, WorkItem *items) {
    __shared__ int64_t s_warp[32][NA];
    __shared__ int64_t s_tot[NA];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int64_t L[NA];
    if (idx < n) item_lengths(m, ids, sizes, mask, idx, L);
    else
        for (int a = 0; a < NA; ++a) L[a] = 0;
    int64_t run[NA];
    for (int a = 0; a < NA; ++a) run[a] = L[a];
    block_scan_na(run, s_warp, s_tot);
    if (idx >= n) return;
    const int64_t *bb = bsum + int64_t(blockIdx.x) * NA;
    int32_t *base[NA] = {arrays_base->vt_off, arrays_base->vt_val, arrays_base->vv_off, arrays_base->vv_val,
                         arrays_base->eu_off, arrays_base->e_w,    arrays_base->et_off, arrays_base->et_val,
                         arrays_base->tt_off, arrays_base->tt_val};
    const int k = ids ? ids[idx] : idx;
    WorkItem w;
    w.k = k;
    w.mask = mask;
    w.blk = m.blk_off[k];
    int32_t *p[NA];
    for (int a = 0; a < NA; ++a) p[a] = base[a] ? base[a] + bb[a] + run[a] : nullptr;
    w.vt_off = p[0]; w.vt_val = p[1]; w.vv_off = p[2]; w.vv_val = p[3];
    w.eu_off = p[4]; w.e_w = p[5]; w.et_off = p[6]; w.et_val = p[7];
    w.tt_off = p[8]; w.tt_val = p[9];
    items[idx] = w;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static int64_t a16(int64_t x) { return (x + 15) & ~int64_t(15); }

static int64_t pow2_at_least(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

Caps caps_of(const ClusterStat &s, const int64_t *sizes) {
    Caps c{};
    c.blk_words = int32_t(blk_words(s.nv_loc, s.n_ext, s.n_own, s.n_halo, s.n_bnd, s.xmap));
    c.nv_own = s.nv_own;
    c.n_vt = s.n_vt;
    c.n_own = s.n_own;
    c.nv_loc = s.nv_loc;
    c.nv_nb = s.nv_nb;
    c.max_deg = s.max_deg;
    c.max_up = s.max_up;
    c.max_e = s.n_e;
    if (sizes) {
        c.max_vv = int32_t(sizes[SZ_VV]);
        c.max_e = int32_t(sizes[SZ_E]);
        c.max_etv = int32_t(sizes[SZ_ET]);
        c.max_tt = int32_t(sizes[SZ_TT]);
    }
    c.hcap = int32_t(std::max<int64_t>(64, pow2_at_least(2 * int64_t(s.n_bnd) + 1)));
    c.n_tot = s.n_ext + s.n_own + s.n_halo;
    c.n_star = s.n_ext + s.n_own;
    return c;
}

int64_t estimate_smem(const ClusterStat &s, int threads) {
    Caps c = caps_of(s, nullptr);
    c.max_vv = 2 * s.n_e;           // each edge is in two VV rows (within the working set, about)
    c.max_etv = s.n_vt + s.n_vt / 2;  // an incidence (x, t) meets 1.5 vertices of t above x on average
    c.max_tt = 4 * s.n_own;
    return plan_smem(c, threads).total;
}

SmemPlan plan_smem(const Caps &c, int threads) {
    SmemPlan p{};
    p.threads = threads;
    p.caps = c;
    const int64_t nwarp = threads / 32;
    const int64_t nvo = c.nv_own;
    p.W = std::max(1, (c.nv_nb + 31) / 32) | 1;  // row stride of the bitmaps (odd)
    p.nch = std::max(1, (c.max_deg + 31) / 32);
    p.pad = int32_t((nvo + 1) & ~int64_t(1));
    int64_t off = 0;
    p.scan = 0;
    off = a16(4 * 128);
    p.blk = int32_t(off);
    off = a16(off + 4 * int64_t(c.blk_words));
    p.vt_off = int32_t(off);
    off = a16(off + 4 * (nvo + 1));
    p.vt_list = int32_t(off);
    off = a16(off + 2 * int64_t(c.n_vt));
    p.c_vv = int32_t(off);
    off = a16(off + 4 * (nvo + 1));
    p.c_e = int32_t(off);
    off = a16(off + 4 * (nvo + 1));
    p.nbr = int32_t(off);
    off = a16(off + 8 * int64_t(c.n_own));
    p.jpos16 = c.max_deg > 256 ? 1 : 0;
    p.jpos = int32_t(off);
    off = a16(off + (p.jpos16 ? 8 : 4) * int64_t(c.n_star));
    // r2: VV staging + upper-endpoint staging, then the edge masks
    p.r2 = int32_t(off);
    p.st_w = int32_t(a16(off + 2 * int64_t(c.max_vv)));
    const int64_t r2 = std::max<int64_t>(4 * int64_t(c.max_e) * p.nch,
                                         a16(2 * int64_t(c.max_vv)) + 2 * int64_t(c.max_e));
    off = a16(off + r2);
    // r1: phase B counters + lane masks | bitmaps + rank prefixes | ET
    // staging | face hash + TT counts + TT staging
    p.r1 = int32_t(off);
    const int64_t cw = a16(2 * nwarp * p.pad);
    p.mk = int32_t(off + cw);
    const int64_t bm = a16(4 * nvo * p.W);
    p.pre = int32_t(off + bm);
    const int64_t hs = a16(4 * int64_t(c.hcap));
    p.tcnt = int32_t(off + hs);
    const int64_t tc = a16(4 * (int64_t(c.n_own) + 1));
    p.st_tt = int32_t(off + hs + tc);
    const int64_t r1 = std::max(std::max(cw + 4 * nwarp * p.pad, bm + nvo * p.W),
                                std::max(2 * int64_t(c.max_etv), hs + tc + 2 * int64_t(c.max_tt)));
    off = a16(off + r1);
    p.total = off > INT32_MAX ? INT32_MAX : int32_t(off);
    return p;
}

int kernel_smem_limit() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

int device_sm_count() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
}

// Largest dynamic shared memory a cluster kernel can be launched with: the
// opt-in limit less the kernels' own static shared memory.
int dynamic_smem_limit() {
    const int optin = kernel_smem_limit();
    int stat = 0;
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, build_kernel<false>) == cudaSuccess) stat = std::max(stat, int(a.sharedSizeBytes));
    if (cudaFuncGetAttributes(&a, build_one_kernel<false>) == cudaSuccess)
        stat = std::max(stat, int(a.sharedSizeBytes));
    if (cudaFuncGetAttributes(&a, count_kernel<false>) == cudaSuccess) stat = std::max(stat, int(a.sharedSizeBytes));
    if (cudaFuncGetAttributes(&a, serve_kernel) == cudaSuccess) stat = std::max(stat, int(a.sharedSizeBytes));
    if (cudaFuncGetAttributes(&a, build_kernel_pi) == cudaSuccess) stat = std::max(stat, int(a.sharedSizeBytes));
    if (cudaFuncGetAttributes(&a, count_kernel_pi) == cudaSuccess) stat = std::max(stat, int(a.sharedSizeBytes));
    if (cudaFuncGetAttributes(&a, build_kernel_team) == cudaSuccess) stat = std::max(stat, int(a.sharedSizeBytes));
    cudaGetLastError();
    return optin - stat;
}

bool prepare_kernels(int smem) {
    // the attribute belongs to the kernel, shared by every context of the
    // process on this device: it only ever grows (a larger limit does not
    // change the occupancy of launches that ask for less)
    static std::mutex mu;
    static int granted[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const int d = dev >= 0 && dev < 64 ? dev : 0;
    smem = std::min(std::max(smem, granted[d]), dynamic_smem_limit());
    bool ok = cudaFuncSetAttribute(build_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
              cudaSuccess;
    ok &= cudaFuncSetAttribute(build_one_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
          cudaSuccess;
    ok &= cudaFuncSetAttribute(count_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
    ok &= cudaFuncSetAttribute(build_kernel_pi, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
    ok &= cudaFuncSetAttribute(count_kernel_pi, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
    ok &= cudaFuncSetAttribute(build_kernel_team, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
    cudaGetLastError();
    if (ok) granted[d] = smem;
    return ok;
}

int max_ctas_per_sm(const SmemPlan &plan, bool spill, bool per_item) {
    int a = 0, b = 0;
    cudaError_t e1, e2;
    if (per_item) {
        e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, build_kernel_pi, plan.threads, plan.total);
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, count_kernel_pi, plan.threads, plan.total);
    } else if (spill) {
        e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, build_kernel<true>, plan.threads, 0);
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, count_kernel<true>, plan.threads, 0);
    } else {
        e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, build_kernel<false>, plan.threads, plan.total);
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, count_kernel<false>, plan.threads, plan.total);
    }
    if (e1 != cudaSuccess || e2 != cudaSuccess) return 0;
    return a < b ? a : b;
}

int max_ctas_per_sm_teams(const SmemPlan &plan, int teams) {
    if (teams < 1 || teams > kMaxTeams || plan.threads % 32 || plan.threads * teams > kMaxTeamBlock) return 0;
    int a = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, build_kernel_team, plan.threads * teams,
                                                      size_t(plan.total) * teams) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return a;
}

int launch_count_pass(const DevMesh &m, const SmemPlan &plan, const int32_t *ids, int32_t n, int64_t *sizes_out,
                      int32_t *err, int32_t *ticket, int grid, void *stream, char *gscratch, uint32_t mask,
                      const SmemPlan *plans) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(ticket, 0, sizeof(int32_t), s);
    if (plans)
        count_kernel_pi<<<grid, plan.threads, plan.total, s>>>(m, plans, ids, n, sizes_out, err, ticket, mask);
    else if (gscratch)
        count_kernel<true><<<grid, plan.threads, 0, s>>>(m, plan, ids, n, sizes_out, err, ticket, gscratch, mask);
    else
        count_kernel<false><<<grid, plan.threads, plan.total, s>>>(m, plan, ids, n, sizes_out, err, ticket, nullptr,
                                                                  mask);
    return int(cudaGetLastError());
}

int bases_scratch_words(int32_t n) { return ((n + kBasesThreads - 1) / kBasesThreads) * NA; }

int launch_bases(const DevMesh &m, const int32_t *ids, int32_t n, const int64_t *sizes, uint32_t mask,
                 const WorkItem *arrays_base, WorkItem *items, int64_t *totals_out, int64_t *bsum, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = (n + kBasesThreads - 1) / kBasesThreads;
    if (nb == 0) return 0;
    bases_sum_kernel<<<nb, kBasesThreads, 0, s>>>(m, ids, n, sizes, mask, bsum);
    bases_scan_kernel<<<1, kBasesThreads, 0, s>>>(nb, bsum, totals_out);
    bases_write_kernel<<<nb, kBasesThreads, 0, s>>>(m, ids, n, sizes, mask, arrays_base, bsum, items);
    return int(cudaGetLastError());
}

int launch_build(const DevMesh &m, const SmemPlan &plan, const WorkItem *items, const int32_t *order, int32_t n,
                 int32_t *err, int32_t *ticket, int grid, void *stream, char *gscratch, const SmemPlan *plans,
                 int teams) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(ticket, 0, sizeof(int32_t), s);
    if (teams > 0) {
        if (plans || gscratch || teams > kMaxTeams || plan.threads * teams > kMaxTeamBlock)
            return int(cudaErrorInvalidValue);
        build_kernel_team<<<grid, plan.threads * teams, size_t(plan.total) * teams, s>>>(m, plan, items, order, n, err,
                                                                                        ticket, plan.threads);
    } else if (plans) build_kernel_pi<<<grid, plan.threads, plan.total, s>>>(m, plans, items, order, n, err, ticket);
    else if (gscratch) build_kernel<true><<<grid, plan.threads, 0, s>>>(m, plan, items, order, n, err, ticket, gscratch);
    else build_kernel<false><<<grid, plan.threads, plan.total, s>>>(m, plan, items, order, n, err, ticket, nullptr);
    return int(cudaGetLastError());
}

// The serving kernel's shared memory limit, grown like the cluster kernels'.
static void grow_serve_attr(int smem) {
    static std::mutex mu;
    static int granted[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const int d = dev >= 0 && dev < 64 ? dev : 0;
    std::lock_guard<std::mutex> lock(mu);
    if (smem <= granted[d]) return;
    if (cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess)
        granted[d] = smem;
    cudaGetLastError();
}

int launch_serve(const DevMesh &m, const SmemPlan &plan, const SmemPlan *plans, const ServeRing &ring, int32_t *err,
                 int grid, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    grow_serve_attr(plan.total);
    serve_kernel<<<grid, plan.threads, plan.total, s>>>(m, plans, ring, err);
    return int(cudaGetLastError());
}

int serve_ctas_per_sm(const SmemPlan &plan) {
    int a = 0;
    grow_serve_attr(plan.total);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, serve_kernel, plan.threads, plan.total) != cudaSuccess)
        return 0;
    return a;
}

int launch_build_one(const DevMesh &m, const SmemPlan &plan, const WorkItem *items, int32_t index, int32_t *err,
                     void *stream, char *gscratch) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (gscratch) build_one_kernel<true><<<1, plan.threads, 0, s>>>(m, plan, items, index, err, gscratch);
    else build_one_kernel<false><<<1, plan.threads, plan.total, s>>>(m, plan, items, index, err, nullptr);
    return int(cudaGetLastError());
}

}  // namespace gale
