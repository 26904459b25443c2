// Producer kernels: per-cluster VT, VV, ET and TT as canonical sorted CSR.
//
// One CTA builds one cluster at a time (persistent CTAs take clusters from a
// ticket counter; the per-cluster baseline launches one CTA per cluster).
// The cluster's working set - its internal tets, its external tets T_ex and
// its face halo (Section 4.3, "Initialization"), stored as 16-bit local rows
// - is copied into shared memory and every relation is built there.  The
// block has one thread per own vertex; per-vertex work is sequential in
// that thread, and every output leaves through shared-memory staging with
// one thread per element (coalesced stores).
//
//  B. VT (Section 4.6 / Algorithm 1: iterate the segment's tets and test
//     each vertex against the segment interval).  Each warp takes a
//     contiguous chunk of the tets (which are in canonical order) and counts
//     its incidences per own vertex; a prefix across warps gives every
//     (warp, vertex) its first slot, and within a warp the lanes holding the
//     same vertex are ranked by a 32-bit lane mask.  Rows come out ascending
//     with no sort.  (The paper's atomicPush, Algorithm 2, fills rows in
//     arbitrary order.)
//  C. VV, ET and most of TT, per own vertex x:
//     - the other vertices of the tets in VT(x) are ORed into a bitmap over
//       the cluster's neighbour universe; local order is canonical order, so
//       the bitmap read in bit order is VV(x) sorted and deduplicated, and
//       its bits above x are the upper endpoints w of the edges (x, w) that x
//       owns; a byte per bitmap word holds the running count of upper bits,
//       so the rank of w is one popcount away;
//     - one block scan of the per-vertex counts places every row;
//     - per upper edge a mask over VT(x) (bit j: the j-th tet contains w):
//       its bits in order are ET(x, w), ascending, and the AND of the masks
//       of (x, w1) and (x, w2) holds the two tets of the face (x, w1, w2), so
//       every face whose lowest vertex is in the cluster gets its TT link.
//  D. TT (Table 1; the paper gives no kernel for it) for the faces (b, c, d)
//     of internal tets (a, b, c, d) with no own vertex: a small
//     open-addressing hash of those faces is probed with the faces of the
//     halo tets.  A face met a third time is reported (non-manifold input).
//
// The counting mode runs the same passes without writes and returns the
// exact sizes the host uses to place outputs and to admit cache entries.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>

#include "gale_internal.h"

namespace gale {

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct Smem {
    int32_t *blk, *scan, *cnt;
    uint16_t *nbr;
    int32_t *vt_off;
    uint16_t *vt_list;
    uint32_t *bmap;   // per own vertex bitmaps (phase B: per-warp counters and masks)
    uint8_t *pre;     // per own vertex, per bitmap word: upper bits in earlier words
    uint16_t *st_ew;  // upper endpoints of the owned edges
    uint32_t *emask;  // per-edge tet masks, then ET row offsets
    uint16_t *st_v;   // VV staging, later ET value staging
    uint32_t *hash;
    int32_t *tcnt;
    int32_t *st_tt;
};

__device__ __forceinline__ Smem carve(char *base, const SmemPlan &p) {
    Smem s;
    s.blk = reinterpret_cast<int32_t *>(base + p.blk);
    s.scan = reinterpret_cast<int32_t *>(base + p.scan);
    s.cnt = reinterpret_cast<int32_t *>(base + p.cnt);
    s.nbr = reinterpret_cast<uint16_t *>(base + p.nbr);
    s.vt_off = reinterpret_cast<int32_t *>(base + p.vt_off);
    s.vt_list = reinterpret_cast<uint16_t *>(base + p.vt_list);
    s.bmap = reinterpret_cast<uint32_t *>(base + p.bmap);
    s.pre = reinterpret_cast<uint8_t *>(base + p.pre);
    s.st_ew = reinterpret_cast<uint16_t *>(base + p.st_ew);
    s.emask = reinterpret_cast<uint32_t *>(base + p.emask);
    s.st_v = reinterpret_cast<uint16_t *>(base + p.emask);
    s.hash = reinterpret_cast<uint32_t *>(base + p.hash);
    s.tcnt = reinterpret_cast<int32_t *>(base + p.tcnt);
    s.st_tt = reinterpret_cast<int32_t *>(base + p.st_tt);
    return s;
}

__device__ __forceinline__ uint32_t vtx(uint2 r, int s) {
    uint32_t w = (s < 2) ? r.x : r.y;
    return (s & 1) ? (w >> 16) : (w & 0xffffu);
}

__device__ __forceinline__ int32_t glob_tet(const BlockHdr &h, const int32_t *tmap, int32_t loc) {
    if (loc < h.n_ext) return tmap[loc];
    if (loc < h.n_ext + h.n_own) return h.t_base + (loc - h.n_ext);
    return tmap[loc - h.n_own];
}

// Bits of `word` (word index q of a bitmap) that stand for local ids > x.
__device__ __forceinline__ uint32_t upper_bits(uint32_t word, int q, int x) {
    const int qx = x >> 5;
    if (q > qx) return word;
    if (q < qx) return 0u;
    const int b = x & 31;
    return b == 31 ? 0u : (word & (FULL << (b + 1)));
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive scan of one value per thread over the block (any multiple of 32
// threads up to 1024); scr needs 33 words.  Two __syncthreads.
__device__ __forceinline__ int block_scan_thread(int v, int32_t *scr, int *total) {
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int incl = warp_incl_scan(v, lane);
    if (lane == 31) scr[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < nw ? scr[lane] : 0;
        const int wi = warp_incl_scan(w, lane);
        if (lane < nw) scr[lane] = wi - w;
        if (lane == 31) scr[32] = wi;
    }
    __syncthreads();
    *total = scr[32];
    return scr[warp] + incl - v;
}

// Exclusive scan in place of a[0..n); returns the total.  Ends synced.
__device__ int block_scan_array(int32_t *a, int n, int32_t *scr) {
    const int NT = blockDim.x;
    const int per = (n + NT - 1) / NT;
    const int b = threadIdx.x * per;
    const int e = min(n, b + per);
    int s = 0;
    for (int i = b; i < e; ++i) s += a[i];
    int total;
    int run = block_scan_thread(s, scr, &total);
    for (int i = b; i < e; ++i) {
        const int v = a[i];
        a[i] = run;
        run += v;
    }
    __syncthreads();
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

__device__ __forceinline__ void cswap(int32_t &a, int32_t &b) {
    const int32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// hash entries: bits [0, 20) = 4 * internal-tet index + slot + 1, bits
// [20, 32) = number of other tets matched to the face
constexpr uint32_t kRefMask = (1u << 20) - 1u;
constexpr uint32_t kMatch = 1u << 20;

// ---------------------------------------------------------------------------
// One cluster.  COUNT: no output writes; sizes -> sizes_out[5].
// `it` points to a shared-memory copy of the work item.
// ---------------------------------------------------------------------------
template <bool COUNT>
__device__ void run_cluster(const DevMesh &m, const SmemPlan &plan, const Smem &S, int64_t blk_word, uint32_t mask,
                            const WorkItem *it, int64_t *sizes_out, int32_t *err) {
    const int NT = blockDim.x, NWARP = NT >> 5;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const Caps &caps = plan.caps;

    // ---------------- A. stage the working set ----------------
    const int32_t *__restrict__ g = m.blocks + blk_word;
    if (tid < kHdrWords) S.blk[tid] = __ldg(g + tid);
    __syncthreads();
    const BlockHdr h = *reinterpret_cast<const BlockHdr *>(S.blk);
    const int64_t words = blk_words(h.nv_loc, h.n_ext, h.n_own, h.n_halo);
    const int W = (h.nv_nb + 31) >> 5;
    const bool fits = words <= caps.blk_words && h.nv_own <= caps.nv_own && h.n_own <= caps.n_own &&
                      h.nv_loc <= caps.nv_loc && h.nv_nb <= caps.nv_nb && h.nv_own >= 0 && h.n_own >= 0 &&
                      h.n_ext >= 0 && h.n_halo >= 0 && h.n_bnd >= 0 && 2 * h.n_bnd + 1 <= caps.hcap &&
                      W <= plan.wp && h.nv_nb <= h.nv_loc;
    if (!fits) {
        if (tid == 0) atomicOr(err, ERR_CAPACITY);
        __syncthreads();
        return;
    }
    {
        const int4 *src = reinterpret_cast<const int4 *>(g);
        int4 *dst = reinterpret_cast<int4 *>(S.blk);
        const int n4 = int(words >> 2);
        for (int i = kHdrWords / 4 + tid; i < n4; i += NT) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    const int32_t *vmap = S.blk + kHdrWords;
    const int32_t *tmap = S.blk + blk_tmap_off(h.nv_loc);
    const uint2 *rows = reinterpret_cast<const uint2 *>(S.blk + blk_rows_off(h.nv_loc, h.n_ext, h.n_halo));
    const int nvo = h.nv_own, lo = h.own_lo;
    const int n_ext = h.n_ext, n_own = h.n_own;
    const int n_vtets = n_ext + n_own;
    const bool want_tt = COUNT || (mask & R_TT);
    const bool do_vv = !COUNT && (mask & R_VV);
    const bool do_et = !COUNT && (mask & R_ET);
    const uint32_t nvo_u = uint32_t(nvo);

    // ---------------- B. VT ----------------
    {
        const int pad = caps.nv_own;
        uint32_t *cw = S.bmap;              // [warp][v]: counts, then next slot
        uint32_t *mk = S.bmap + NWARP * pad;  // [warp][v]: lanes holding v
        const int chunk = ((n_vtets + NWARP - 1) / NWARP + 31) & ~31;
        const int c0 = min(n_vtets, warp * chunk), c1 = min(n_vtets, c0 + chunk);
        for (int i = tid; i < 2 * NWARP * pad; i += NT) S.bmap[i] = 0u;
        __syncthreads();
        for (int i = c0 + lane; i < c1; i += 32) {
            const uint2 r = rows[i];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const uint32_t d = vtx(r, s) - uint32_t(lo);
                if (d < nvo_u) atomicAdd(&cw[warp * pad + d], 1u);
            }
        }
        __syncthreads();
        // row lengths -> offsets; every (warp, vertex) gets its first slot
        for (int v = tid; v < nvo; v += NT) {
            int tot = 0;
            for (int w = 0; w < NWARP; ++w) tot += int(cw[w * pad + v]);
            S.vt_off[v] = tot;
        }
        __syncthreads();
        const int vt_total = block_scan_array(S.vt_off, nvo, S.scan);
        bool bad = vt_total > caps.n_vt;
        for (int v = tid; v < nvo; v += NT) {
            int run = S.vt_off[v];
            const int d = (v + 1 < nvo ? S.vt_off[v + 1] : vt_total) - run;
            bad |= d > caps.max_deg;
            for (int w = 0; w < NWARP; ++w) {
                const int c = int(cw[w * pad + v]);
                cw[w * pad + v] = uint32_t(run);
                run += c;
            }
        }
        if (tid == 0) S.vt_off[nvo] = vt_total;
        if (__syncthreads_or(bad)) {
            if (tid == 0) atomicOr(err, ERR_CAPACITY);
            return;
        }
        if (!bad) {
            // fill in tet order, 32 tets per step of each warp
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
                        S.vt_list[cw[warp * pad + d[s]] + __popc(mm[s] & lt)] = uint16_t(i);
                    }
                }
                __syncwarp();
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    if (d[s] < nvo_u && (mm[s] & lt) == 0u) {
                        cw[warp * pad + d[s]] += uint32_t(__popc(mm[s]));
                        mk[warp * pad + d[s]] = 0u;
                    }
                __syncwarp();
            }
        }
        __syncthreads();
        if (COUNT) {
            if (tid == 0) sizes_out[SZ_VT] = vt_total;
        } else if (mask & R_VT) {
            for (int i = tid; i <= nvo; i += NT) it->vt_off[i] = S.vt_off[i];
            for (int j = tid; j < vt_total; j += NT) it->vt_val[j] = glob_tet(h, tmap, S.vt_list[j]);
        }
    }
    if (!(COUNT || do_vv || do_et || want_tt)) return;

    // ---------------- C. VV, ET and TT faces with an own lowest vertex ----
    int32_t *c_vv = S.cnt, *c_e = S.cnt + caps.nv_own, *c_et = S.cnt + 2 * caps.nv_own;
    __syncthreads();  // phase B counters and masks are dead
    if (want_tt) {
        uint32_t *nb32 = reinterpret_cast<uint32_t *>(S.nbr);
        for (int i = tid; i < 2 * n_own; i += NT) nb32[i] = 0xffffffffu;
    }
    // pass 1: bitmaps and counts
    for (int i = tid; i < nvo; i += NT) {
        const int x = lo + i;
        const int beg = S.vt_off[i], L = S.vt_off[i + 1] - beg;
        uint32_t *bm = S.bmap + i * plan.wp;
        for (int q = 0; q < W; ++q) bm[q] = 0u;
        int etv = 0;
        for (int j0 = 0; j0 < L; j0 += 4) {
            uint2 r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) r[u] = rows[S.vt_list[beg + min(j0 + u, L - 1)]];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (j0 + u < L) {
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const uint32_t y = vtx(r[u], s);
                        if (int(y) != x) atomicOr(&bm[y >> 5], 1u << (y & 31));
                        etv += int(y) > x;
                    }
                }
            }
        }
        int vv = 0, ec = 0;
        uint8_t *pr = S.pre + i * plan.wp;
        for (int q = 0; q < W; ++q) {
            const uint32_t word = bm[q];
            pr[q] = uint8_t(ec);
            vv += __popc(word);
            ec += __popc(upper_bits(word, q, x));
        }
        c_vv[i] = vv;
        c_e[i] = ec;
        c_et[i] = etv;
    }
    __syncthreads();
    const int tot_vv = block_scan_array(c_vv, nvo, S.scan);
    const int tot_e = block_scan_array(c_e, nvo, S.scan);
    const int tot_et = block_scan_array(c_et, nvo, S.scan);
    if (COUNT && tid == 0) {
        sizes_out[SZ_VV] = tot_vv;
        sizes_out[SZ_E] = tot_e;
        sizes_out[SZ_ET] = tot_et;
    }
    if (tot_e > caps.max_e || (do_vv && tot_vv > caps.max_vv) || (do_et && tot_et > caps.max_etv)) {
        if (tid == 0) atomicOr(err, ERR_CAPACITY);
        return;
    }
    // pass 2: VV rows and the upper endpoints of the owned edges, staged
    bool bad_up = false;
    for (int i = tid; i < nvo; i += NT) {
        const int x = lo + i;
        uint32_t *bm = S.bmap + i * plan.wp;
        int p = c_vv[i], e = c_e[i];
        const int e_end = (i + 1 < nvo) ? c_e[i + 1] : tot_e;
        bad_up |= (e_end - e) > caps.max_up || (e_end - e) > 255;
        for (int q = 0; q < W; ++q) {
            uint32_t word = bm[q];
            uint32_t up = upper_bits(word, q, x);
            bm[q] = up;  // from here on the bitmap holds the upper neighbours only
            if (do_vv)
                while (word) {
                    const int b = __ffs(word) - 1;
                    word &= word - 1;
                    S.st_v[p++] = uint16_t(q * 32 + b);
                }
            while (up) {
                const int b = __ffs(up) - 1;
                up &= up - 1;
                S.st_ew[e++] = uint16_t(q * 32 + b);
            }
        }
    }
    if (__syncthreads_or(bad_up)) {
        if (tid == 0) atomicOr(err, ERR_CAPACITY);
        return;
    }
    if (do_vv) {
        for (int i = tid; i < nvo; i += NT) it->vv_off[i] = c_vv[i];
        if (tid == 0) it->vv_off[nvo] = tot_vv;
        for (int j = tid; j < tot_vv; j += NT) it->vv_val[j] = vmap[S.st_v[j]];
    }
    if (do_et) {
        for (int i = tid; i < nvo; i += NT) it->eu_off[i] = c_e[i];
        if (tid == 0) {
            it->eu_off[nvo] = tot_e;
            it->et_off[tot_e] = tot_et;
        }
        for (int e = tid; e < tot_e; e += NT) it->e_w[e] = vmap[S.st_ew[e]];
    }
    if (!(do_et || want_tt)) return;
    __syncthreads();  // VV staging is dead: the edge masks take its place
    {
        // pass 3a: per-edge tet masks and TT links
        const int nch = plan.nch;
        int32_t flags = 0;
        for (int i = tid; i < nvo; i += NT) {
            const int x = lo + i;
            const int beg = S.vt_off[i], L = S.vt_off[i + 1] - beg;
            const int e0 = c_e[i], E = ((i + 1 < nvo) ? c_e[i + 1] : tot_e) - e0;
            const uint32_t *bm = S.bmap + i * plan.wp;
            const uint8_t *pr = S.pre + i * plan.wp;
            uint32_t *em = S.emask + e0 * nch;  // em[r * nch + c]
            for (int q = 0; q < E * nch; ++q) em[q] = 0u;
            // rank of an upper neighbour y among x's upper neighbours
            auto rank = [&](uint32_t y) -> int {
                const int q = int(y >> 5);
                return int(pr[q]) + __popc(bm[q] & ((1u << (y & 31)) - 1u));
            };
            for (int j0 = 0; j0 < L; j0 += 4) {
                uint2 r[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) r[u] = rows[S.vt_list[beg + min(j0 + u, L - 1)]];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u;
                    if (j < L) {
#pragma unroll
                        for (int s = 1; s < 4; ++s) {
                            const uint32_t y = vtx(r[u], s);
                            if (int(y) > x) atomicOr(&em[rank(y) * nch + (j >> 5)], 1u << (j & 31));
                        }
                    }
                }
            }
            if (!want_tt) continue;
            // faces (x, w1, w2) with x lowest: the tets are the bits of
            // em[w1] & em[w2]; links are kept for internal tets
            for (int j0 = 0; j0 < L; j0 += 4) {
                int tl[4];
                uint2 r[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) tl[u] = S.vt_list[beg + min(j0 + u, L - 1)];
#pragma unroll
                for (int u = 0; u < 4; ++u) r[u] = rows[tl[u]];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u;
                    const uint32_t io = uint32_t(tl[u] - n_ext);
                    if (j >= L || io >= uint32_t(n_own)) continue;
                    const int p = (int(vtx(r[u], 0)) == x) ? 0 : (int(vtx(r[u], 1)) == x) ? 1 : 2;
                    if (p >= 2) continue;
                    int rk[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int s2 = 1; s2 < 4; ++s2)
                        if (s2 > p) rk[s2] = rank(vtx(r[u], s2));
#pragma unroll
                    for (int a = 1; a < 4; ++a)
#pragma unroll
                        for (int b2 = a + 1; b2 < 4; ++b2) {
                            if (a <= p) continue;
                            const int opp = 6 - p - a - b2;  // the slot outside {p, a, b2}
                            int partner = -1, found = 0;
                            for (int c = 0; c < nch; ++c) {
                                uint32_t mk2 = em[rk[a] * nch + c] & em[rk[b2] * nch + c];
                                if (c == (j >> 5)) mk2 &= ~(1u << (j & 31));
                                found += __popc(mk2);
                                if (mk2 && partner < 0) partner = 32 * c + __ffs(mk2) - 1;
                            }
                            if (found > 1) flags |= ERR_NONMANIFOLD;
                            if (partner >= 0) S.nbr[io * 4 + opp] = S.vt_list[beg + partner];
                        }
                }
            }
        }
        if (flags) atomicOr(err, flags);
        __syncthreads();  // bitmaps are dead: the ET value staging takes their place
        if (do_et) {
            // pass 3b: ET rows from the masks; each edge's first mask word
            // then holds its row offset for the copy-out
            uint16_t *st_et = reinterpret_cast<uint16_t *>(S.bmap);
            for (int i = tid; i < nvo; i += NT) {
                const int beg = S.vt_off[i];
                const int e0 = c_e[i], E = ((i + 1 < nvo) ? c_e[i + 1] : tot_e) - e0;
                uint32_t *em = S.emask + e0 * nch;
                int t = c_et[i];
                for (int rr = 0; rr < E; ++rr) {
                    const int t0 = t;
                    for (int c = 0; c < nch; ++c) {
                        uint32_t mk2 = em[rr * nch + c];
                        while (mk2) {
                            const int b = __ffs(mk2) - 1;
                            mk2 &= mk2 - 1;
                            st_et[t++] = S.vt_list[beg + 32 * c + b];
                        }
                    }
                    em[rr * nch] = uint32_t(t0);
                }
            }
            __syncthreads();
            for (int e = tid; e < tot_e; e += NT) it->et_off[e] = int32_t(S.emask[e * nch]);
            for (int j = tid; j < tot_et; j += NT) it->et_val[j] = glob_tet(h, tmap, st_et[j]);
        }
        __syncthreads();
    }

    if (want_tt) {
        // ---------------- D. faces with no own vertex, against the halo ----
        const uint32_t hmask = uint32_t(caps.hcap - 1);
        uint32_t *hash = S.hash;
        for (int i = tid; i < caps.hcap; i += NT) hash[i] = 0u;
        __syncthreads();
        int32_t flags = 0;
        for (int i = tid; i < n_own; i += NT) {
            const uint2 r = rows[n_ext + i];
            if (vtx(r, 1) - uint32_t(lo) < nvo_u) continue;  // face (b, c, d) has an own vertex
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
        __syncthreads();
        const int n_halo = h.n_halo;
        for (int j = tid; j < n_halo; j += NT) {
            const int tl = n_vtets + j;
            const uint2 r = rows[tl];
            for (int s = 0; s < 4; ++s) {
                const uint64_t key = face_key(r, s);
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
        }
        if (flags) atomicOr(err, flags);
        __syncthreads();
        // counts per internal tet -> offsets
        int32_t *tcnt = S.tcnt;
        for (int i = tid; i < n_own; i += NT) {
            const uint2 nb = *reinterpret_cast<const uint2 *>(&S.nbr[i * 4]);
            tcnt[i] = ((nb.x & 0xffffu) != 0xffffu) + ((nb.x >> 16) != 0xffffu) + ((nb.y & 0xffffu) != 0xffffu) +
                      ((nb.y >> 16) != 0xffffu);
        }
        __syncthreads();
        const int tot_tt = block_scan_array(tcnt, n_own, S.scan);
        if (COUNT) {
            if (tid == 0) sizes_out[SZ_TT] = tot_tt;
        } else {
            if (tot_tt > caps.max_tt) {
                if (tid == 0) atomicOr(err, ERR_CAPACITY);
                return;
            }
            for (int i = tid; i < n_own; i += NT) {
                const uint2 nb = *reinterpret_cast<const uint2 *>(&S.nbr[i * 4]);
                const uint32_t n0 = nb.x & 0xffffu, n1 = nb.x >> 16, n2 = nb.y & 0xffffu, n3 = nb.y >> 16;
                // absent neighbours sort last as INT32_MAX
                int32_t v0 = n0 != 0xffffu ? glob_tet(h, tmap, int32_t(n0)) : INT32_MAX;
                int32_t v1 = n1 != 0xffffu ? glob_tet(h, tmap, int32_t(n1)) : INT32_MAX;
                int32_t v2 = n2 != 0xffffu ? glob_tet(h, tmap, int32_t(n2)) : INT32_MAX;
                int32_t v3 = n3 != 0xffffu ? glob_tet(h, tmap, int32_t(n3)) : INT32_MAX;
                cswap(v0, v1); cswap(v2, v3); cswap(v0, v2); cswap(v1, v3); cswap(v1, v2);
                const int p = tcnt[i];
                it->tt_off[i] = p;
                int32_t *o = S.st_tt + p;
                if (v0 != INT32_MAX) o[0] = v0;
                if (v1 != INT32_MAX) o[1] = v1;
                if (v2 != INT32_MAX) o[2] = v2;
                if (v3 != INT32_MAX) o[3] = v3;
            }
            if (tid == 0) it->tt_off[n_own] = tot_tt;
            __syncthreads();
            for (int j = tid; j < tot_tt; j += NT) it->tt_val[j] = S.st_tt[j];
        }
    }
    __syncthreads();
}

// SPILL: the cluster's regions live in a per-CTA slice of global scratch
// (clusters whose working set exceeds shared memory); otherwise in dynamic
// shared memory.
template <bool SPILL>
__device__ __forceinline__ char *region_base(char *smem, char *gscratch, const SmemPlan &plan) {
    return SPILL ? gscratch + size_t(blockIdx.x) * size_t(plan.total) : smem;
}

// Blocks have up to 1024 threads (one per own vertex), so every cluster
// kernel is bounded to 64 registers per thread.
constexpr int kMaxThreads = 1024;

template <bool SPILL>
__global__ void __launch_bounds__(kMaxThreads) count_kernel(DevMesh m, SmemPlan plan, const int32_t *ids, int32_t n, int64_t *sizes, int32_t *err,
                             int32_t *ticket, char *gscratch) {
    extern __shared__ __align__(16) char smem[];
    const Smem S = carve(region_base<SPILL>(smem, gscratch, plan), plan);
    __shared__ int32_t s_idx;
    __shared__ int64_t s_sizes[SZ_N];
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(ticket, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= n) break;
        const int k = ids ? ids[idx] : idx;
        if (k < 0 || k >= m.K) {
            if (threadIdx.x == 0) atomicOr(err, ERR_BAD_ITEM);
            continue;
        }
        if (threadIdx.x < SZ_N) s_sizes[threadIdx.x] = 0;
        __syncthreads();
        run_cluster<true>(m, plan, S, m.blk_off[k], 0u, nullptr, s_sizes, err);
        __syncthreads();
        if (threadIdx.x < SZ_N) sizes[int64_t(k) * SZ_N + threadIdx.x] = s_sizes[threadIdx.x];
    }
}

template <bool SPILL>
__global__ void __launch_bounds__(kMaxThreads) build_kernel(DevMesh m, SmemPlan plan, const WorkItem *items, const int32_t *order, int32_t n,
                             int32_t *err, int32_t *ticket, char *gscratch) {
    extern __shared__ __align__(16) char smem[];
    const Smem S = carve(region_base<SPILL>(smem, gscratch, plan), plan);
    __shared__ int32_t s_idx;
    __shared__ WorkItem s_item;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(ticket, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= n) break;
        if (threadIdx.x == 0) s_item = items[order ? order[idx] : idx];
        __syncthreads();
        const int k = s_item.k;
        if (k < 0 || k >= m.K) {
            if (threadIdx.x == 0) atomicOr(err, ERR_BAD_ITEM);
            continue;
        }
        run_cluster<false>(m, plan, S, s_item.blk, s_item.mask, &s_item, nullptr, err);
    }
}

template <bool SPILL>
__global__ void __launch_bounds__(kMaxThreads) build_one_kernel(DevMesh m, SmemPlan plan, const WorkItem *items, int32_t index, int32_t *err,
                                 char *gscratch) {
    extern __shared__ __align__(16) char smem[];
    const Smem S = carve(region_base<SPILL>(smem, gscratch, plan), plan);
    __shared__ WorkItem s_item;
    if (threadIdx.x == 0) s_item = items[index];
    __syncthreads();
    if (s_item.k < 0 || s_item.k >= m.K) {
        if (threadIdx.x == 0) atomicOr(err, ERR_BAD_ITEM);
        return;
    }
    run_cluster<false>(m, plan, S, s_item.blk, s_item.mask, &s_item, nullptr, err);
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

__global__ void __launch_bounds__(1024) serve_kernel(DevMesh m, SmemPlan plan, ServeRing ring, int32_t *err) {
    extern __shared__ __align__(16) char smem[];
    const Smem S = carve(smem, plan);
    __shared__ long long s_t;
    __shared__ WorkItem s_item;
    unsigned long long last = globaltimer();
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
                if (sleep_ns < 8192) sleep_ns *= 2;
            }
            if (t >= 0) {
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
        if (s_item.k >= 0 && s_item.k < m.K)
            run_cluster<false>(m, plan, S, s_item.blk, s_item.mask, &s_item, nullptr, err);
        else if (threadIdx.x == 0)
            atomicOr(err, ERR_BAD_ITEM);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence_system();
            st_release_sys(ring.done + (t % ring.cap), t);
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
    const int64_t nvo = m.I_V[k + 1] - m.I_V[k];
    const int64_t nown = m.I_T[k + 1] - m.I_T[k];
    const bool vt = mask & R_VT, vv = mask & R_VV, et = mask & R_ET, tt = mask & R_TT;
    L[0] = vt ? nvo + 1 : 0;
    L[1] = vt ? sz[SZ_VT] : 0;
    L[2] = vv ? nvo + 1 : 0;
    L[3] = vv ? sz[SZ_VV] : 0;
    L[4] = et ? nvo + 1 : 0;
    L[5] = et ? sz[SZ_E] : 0;
    L[6] = et ? sz[SZ_E] + 1 : 0;
    L[7] = et ? sz[SZ_ET] : 0;
    L[8] = tt ? nown + 1 : 0;
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

SmemPlan plan_smem(const Caps &c, int threads) {
    SmemPlan p{};
    p.threads = threads;
    p.caps = c;
    const int nwarp = threads / 32;
    const int W = (c.nv_nb + 31) / 32;
    p.nch = std::max(1, (c.max_deg + 31) / 32);
    p.wp = std::max(W, 1) | 1;
    int64_t off = 0;
    p.blk = 0;
    off = a16(int64_t(4) * c.blk_words);
    p.scan = int32_t(off);
    off = a16(off + 4 * 40);
    p.cnt = int32_t(off);
    off = a16(off + 4 * 3 * int64_t(c.nv_own));
    p.nbr = int32_t(off);
    off = a16(off + 8 * int64_t(c.n_own));
    p.vt_off = int32_t(off);
    off = a16(off + 4 * (int64_t(c.nv_own) + 1));
    p.vt_list = int32_t(off);
    off = a16(off + 2 * int64_t(c.n_vt));
    p.bmap = int32_t(off);
    // phase B: per-warp counters and masks; phase C: per-vertex bitmaps and
    // their rank prefixes, later the ET value staging
    const int64_t bm_b = 8 * int64_t(nwarp) * c.nv_own;
    const int64_t bm_c = a16(4 * int64_t(c.nv_own) * p.wp) + int64_t(c.nv_own) * p.wp;
    const int64_t st_et = 2 * int64_t(c.max_etv);
    p.pre = int32_t(off + a16(4 * int64_t(c.nv_own) * p.wp));
    off = a16(off + std::max(bm_b, std::max(bm_c, st_et)));
    p.st_ew = int32_t(off);
    off = a16(off + 2 * int64_t(c.max_e));
    // VV staging, later the per-edge tet masks
    p.emask = int32_t(off);
    p.st_v = p.emask;
    const int64_t end_c = a16(off + std::max<int64_t>(4 * int64_t(c.max_e) * p.nch, 2 * int64_t(c.max_vv)));
    // phase D overlays from vt_off (cnt and nbr stay)
    p.hash = p.vt_off;
    p.tcnt = int32_t(a16(int64_t(p.hash) + 4 * int64_t(c.hcap)));
    p.st_tt = int32_t(a16(int64_t(p.tcnt) + 4 * (int64_t(c.n_own) + 1)));
    const int64_t end_d = a16(int64_t(p.st_tt) + 4 * int64_t(c.max_tt));
    const int64_t tot = std::max(end_c, end_d);
    p.total = tot > INT32_MAX ? INT32_MAX : int32_t(tot);
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

void prepare_kernels(int smem) {
    cudaFuncSetAttribute(build_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(build_one_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(count_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

int max_ctas_per_sm(const SmemPlan &plan, bool spill) {
    int a = 0, b = 0;
    cudaError_t e1, e2;
    if (spill) {
        e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, build_kernel<true>, plan.threads, 0);
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, count_kernel<true>, plan.threads, 0);
    } else {
        e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, build_kernel<false>, plan.threads, plan.total);
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, count_kernel<false>, plan.threads, plan.total);
    }
    if (e1 != cudaSuccess || e2 != cudaSuccess) return 0;
    return a < b ? a : b;
}

int launch_count_pass(const DevMesh &m, const SmemPlan &plan, const int32_t *ids, int32_t n, int64_t *sizes_out,
                      int32_t *err, int32_t *ticket, int grid, void *stream, char *gscratch) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(ticket, 0, sizeof(int32_t), s);
    if (gscratch) count_kernel<true><<<grid, plan.threads, 0, s>>>(m, plan, ids, n, sizes_out, err, ticket, gscratch);
    else count_kernel<false><<<grid, plan.threads, plan.total, s>>>(m, plan, ids, n, sizes_out, err, ticket, nullptr);
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
                 int32_t *err, int32_t *ticket, int grid, void *stream, char *gscratch) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(ticket, 0, sizeof(int32_t), s);
    if (gscratch) build_kernel<true><<<grid, plan.threads, 0, s>>>(m, plan, items, order, n, err, ticket, gscratch);
    else build_kernel<false><<<grid, plan.threads, plan.total, s>>>(m, plan, items, order, n, err, ticket, nullptr);
    return int(cudaGetLastError());
}

int launch_serve(const DevMesh &m, const SmemPlan &plan, const ServeRing &ring, int32_t *err, int grid,
                 void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.total);
    serve_kernel<<<grid, plan.threads, plan.total, s>>>(m, plan, ring, err);
    return int(cudaGetLastError());
}

int serve_ctas_per_sm(const SmemPlan &plan) {
    int a = 0;
    cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.total);
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
