// Producer kernels: per-cluster VT, VV, ET and TT as canonical sorted CSR.
//
// One CTA builds one cluster at a time (persistent CTAs take clusters from a
// ticket counter).  The cluster's working set - its internal tets, its
// external tets T_ex and its face halo (Section 4.3, "Initialization"),
// stored as 16-bit local rows - is copied into shared memory, and every
// relation is built there:
//
//  B. VT (Section 4.6: iterate the segment's tets, test each vertex against
//     the segment interval I_V, Algorithm 1).  Counts per own vertex by
//     shared-memory atomics, an exclusive scan, then a deterministic fill:
//     tets are taken in windows of one tet per thread; each warp ORs a
//     32-bit presence mask per own vertex, and each vertex's thread walks
//     the masks in (warp, lane) order, so every row comes out ascending
//     without a sort.  The paper's atomicPush (Algorithm 2) gives rows in
//     arbitrary order; this fill gives the canonical one.
//  C. VV and ET, one warp per own vertex x: the other vertices of the tets
//     in VT(x) are ORed into a bitmap over the cluster's local vertices
//     (local order = canonical order, so reading the bitmap in bit order
//     yields VV(x) sorted and deduplicated).  The bits above x are the edges
//     (x, w) x owns; the rank of w among them comes from a popcount prefix.
//     Each tet ORs its lane bit into the mask of each of its edges, so the
//     position of tet j in ET(x, w) is the popcount of the lanes below j:
//     rows come out sorted by (w, t).  Warps of a chunk of NWARP vertices
//     get their output positions from one block scan.
//  D. TT (Table 1; never described by the paper): the faces of the internal
//     tets go into an open-addressing hash keyed by their three local
//     vertex ids; a second internal tet with the same face links the pair,
//     and the faces of the external and halo tets are probed to link the
//     rest.  A face met a third time is reported (non-manifold input).
//
// Outputs are written with one thread per element of a contiguous range
// (VT) or by warps over their vertex's contiguous range (VV, ET), so stores
// are coalesced; the counting mode runs the same passes without writes and
// returns the exact sizes used for output placement.
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <type_traits>

#include "gale_internal.h"

namespace gale {

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct Smem {
    int32_t *blk;
    int32_t *scan;
    int32_t *vt_off;
    int32_t *cur;
    uint16_t *vt_list;
    uint32_t *uni;
    uint32_t *hash;
    uint32_t *nbr;
};

__device__ __forceinline__ Smem carve(char *base, const SmemPlan &p) {
    Smem s;
    s.blk = reinterpret_cast<int32_t *>(base + p.blk);
    s.scan = reinterpret_cast<int32_t *>(base + p.scan);
    s.vt_off = reinterpret_cast<int32_t *>(base + p.vt_off);
    s.cur = reinterpret_cast<int32_t *>(base + p.cur);
    s.vt_list = reinterpret_cast<uint16_t *>(base + p.vt_list);
    s.uni = reinterpret_cast<uint32_t *>(base + p.uni);
    s.hash = reinterpret_cast<uint32_t *>(base + p.hash);
    s.nbr = reinterpret_cast<uint32_t *>(base + p.nbr);
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
    int qx = x >> 5;
    if (q > qx) return word;
    if (q < qx) return 0u;
    int b = x & 31;
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

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Exclusive scan of one value per thread over the block; returns the
// thread's prefix, total in *total.  scr needs NWARP+1 words.  Contains
// two __syncthreads.
template <int NT>
__device__ __forceinline__ int block_scan_thread(int v, int32_t *scr, int *total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = warp_incl_scan(v, lane);
    if (lane == 31) scr[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NW ? scr[lane] : 0;
        int wi = warp_incl_scan(w, lane);
        if (lane < NW) scr[lane] = wi - w;
        if (lane == NW - 1) scr[NW] = wi;
    }
    __syncthreads();
    int r = scr[warp] + incl - v;
    *total = scr[NW];
    return r;
}

// Exclusive scan in place of a[0..n) (n small); returns the total.
template <int NT>
__device__ int block_scan_array(int32_t *a, int n, int32_t *scr) {
    const int per = (n + NT - 1) / NT;
    const int b = threadIdx.x * per;
    const int e = min(n, b + per);
    int s = 0;
    for (int i = b; i < e; ++i) s += a[i];
    int total;
    int run = block_scan_thread<NT>(s, scr, &total);
    for (int i = b; i < e; ++i) {
        int v = a[i];
        a[i] = run;
        run += v;
    }
    __syncthreads();
    return total;
}

__device__ __forceinline__ uint64_t face_key(uint2 r, int s) {
    // the three vertices of the row other than slot s, ascending, packed as
    // 16-bit fields: drop field s of the packed 64-bit row
    const uint64_t row = uint64_t(r.x) | (uint64_t(r.y) << 32);
    const int sh = 16 * s;
    const uint64_t low = sh ? (row & ((uint64_t(1) << sh) - 1)) : 0ull;
    const uint64_t high = s == 3 ? 0ull : ((row >> (sh + 16)) << sh);
    return low | high;
}

__device__ __forceinline__ uint32_t face_hash(uint64_t key, uint32_t mask) {
    return uint32_t((key * 0x9E3779B97F4A7C15ull) >> 32) & mask;
}

__device__ __forceinline__ void cswap(int32_t &a, int32_t &b) {
    const int32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// sorting network for 4 values held in registers
__device__ __forceinline__ void sort4_net(int32_t &a, int32_t &b, int32_t &c, int32_t &d) {
    cswap(a, b); cswap(c, d); cswap(a, c); cswap(b, d); cswap(b, c);
}

// ---------------------------------------------------------------------------
// One cluster.  COUNT: no output writes, sizes -> sizes_out[5].
// ---------------------------------------------------------------------------
template <int NT, bool COUNT>
__device__ void run_cluster(const DevMesh &m, const SmemPlan &plan, const Smem &S, int64_t blk_word, uint32_t mask,
                            const WorkItem *it, int64_t *sizes_out, int32_t *err) {
    constexpr int NWARP = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Caps &caps = plan.caps;

    // ---------------- A. stage the working set ----------------
    const int32_t *g = m.blocks + blk_word;
    if (tid < 8) S.blk[tid] = __ldg(g + tid);
    __syncthreads();
    const BlockHdr h = *reinterpret_cast<const BlockHdr *>(S.blk);
    const int64_t words = blk_words(h.nv_loc, h.n_ext, h.n_own, h.n_halo);
    const int W = (h.nv_loc + 31) >> 5;
    const bool fits = words <= caps.blk_words && h.nv_own <= caps.nv_own && h.n_own <= caps.n_own &&
                      h.nv_loc <= caps.nv_loc && h.nv_own >= 0 && h.n_own >= 0 &&
                      int64_t(4) * h.n_own + 1 <= caps.hcap;
    if (!fits) {
        if (tid == 0) atomicOr(err, ERR_CAPACITY);
        __syncthreads();
        return;
    }
    {
        const int4 *src = reinterpret_cast<const int4 *>(g);
        int4 *dst = reinterpret_cast<int4 *>(S.blk);
        const int n4 = int(words >> 2);
        for (int i = 2 + tid; i < n4; i += NT) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    const int32_t *vmap = S.blk + 8;
    const int32_t *tmap = S.blk + blk_tmap_off(h.nv_loc);
    const uint2 *rows = reinterpret_cast<const uint2 *>(S.blk + blk_rows_off(h.nv_loc, h.n_ext, h.n_halo));
    const int nvo = h.nv_own, lo = h.own_lo;
    const int n_vtets = h.n_ext + h.n_own;

    const bool need_vt = COUNT || (mask & (R_VT | R_VV | R_ET));
    int vt_total = 0;
    if (need_vt) {
        // ---------------- B. VT ----------------
        for (int i = tid; i < nvo; i += NT) S.cur[i] = 0;
        __syncthreads();
        for (int i = tid; i < n_vtets; i += NT) {
            uint2 r = rows[i];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                uint32_t d = vtx(r, s) - uint32_t(lo);
                if (d < uint32_t(nvo)) atomicAdd(&S.cur[d], 1);
            }
        }
        __syncthreads();
        for (int i = tid; i < nvo; i += NT) S.vt_off[i] = S.cur[i];
        __syncthreads();
        vt_total = block_scan_array<NT>(S.vt_off, nvo, S.scan);
        bool bad = vt_total > caps.n_vt;
        for (int i = tid; i < nvo; i += NT) {
            S.cur[i] = S.vt_off[i];
            int deg = (i + 1 < nvo ? S.vt_off[i + 1] : vt_total) - S.vt_off[i];
            if (deg > caps.max_deg) bad = true;
        }
        if (tid == 0) S.vt_off[nvo] = vt_total;
        if (__syncthreads_or(bad)) {
            if (tid == 0) atomicOr(err, ERR_CAPACITY);
            return;
        }
        // windowed presence masks, masks[w * pad + v]
        uint32_t *masks = S.uni;
        const int pad = caps.nv_own;
        for (int i = tid; i < NWARP * pad; i += NT) masks[i] = 0;
        __syncthreads();
        for (int base = 0; base < n_vtets; base += NT) {
            const int i = base + tid;
            if (i < n_vtets) {
                uint2 r = rows[i];
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    uint32_t d = vtx(r, s) - uint32_t(lo);
                    if (d < uint32_t(nvo)) atomicOr(&masks[warp * pad + d], 1u << lane);
                }
            }
            __syncthreads();
            for (int v = tid; v < nvo; v += NT) {
                int c = S.cur[v];
                for (int w = 0; w < NWARP; ++w) {
                    uint32_t mk = masks[w * pad + v];
                    if (mk) {
                        masks[w * pad + v] = 0;
                        const int tb = base + w * 32;
                        do {
                            int b = __ffs(mk) - 1;
                            mk &= mk - 1;
                            S.vt_list[c++] = uint16_t(tb + b);
                        } while (mk);
                    }
                }
                S.cur[v] = c;
            }
            __syncthreads();
        }
        if (COUNT) {
            if (tid == 0) sizes_out[SZ_VT] = vt_total;
        } else if (mask & R_VT) {
            for (int i = tid; i <= nvo; i += NT) it->vt_off[i] = S.vt_off[i];
            for (int j = tid; j < vt_total; j += NT) it->vt_val[j] = glob_tet(h, tmap, S.vt_list[j]);
        }
    }

    if (COUNT || (mask & (R_VV | R_ET))) {
        // ---------------- C. VV and ET ----------------
        const int Wc = (caps.nv_loc + 31) >> 5;
        uint32_t *bm = S.uni + warp * plan.warp_words;
        int32_t *pre = reinterpret_cast<int32_t *>(bm + Wc);
        uint32_t *emask = bm + 2 * Wc;
        int32_t *ecnt = reinterpret_cast<int32_t *>(emask + caps.max_up);
        int32_t *scnt = S.scan + (NWARP + 1);       // [NWARP][3]
        int32_t *sbase = scnt + 3 * NWARP;          // [NWARP][3]
        int32_t *carry = sbase + 3 * NWARP;         // [3]
        if (tid < 3) carry[tid] = 0;
        __syncthreads();
        const bool do_vv = !COUNT && (mask & R_VV);
        const bool do_et = !COUNT && (mask & R_ET);
        for (int r0 = 0; r0 < nvo; r0 += NWARP) {
            const int i = r0 + warp;
            const bool active = i < nvo;
            const int x = lo + i;
            int vvc = 0, ec = 0, etv = 0, beg = 0, L = 0;
            bool bad = false;
            if (active) {
                beg = S.vt_off[i];
                L = S.vt_off[i + 1] - beg;
                for (int q = lane; q < W; q += 32) bm[q] = 0;
                __syncwarp();
                for (int j = lane; j < L; j += 32) {
                    uint2 r = rows[S.vt_list[beg + j]];
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        uint32_t y = vtx(r, s);
                        if (int(y) != x) atomicOr(&bm[y >> 5], 1u << (y & 31));
                        etv += int(y) > x;
                    }
                }
                __syncwarp();
                int run = 0;
                for (int q0 = 0; q0 < W; q0 += 32) {
                    const int q = q0 + lane;
                    uint32_t word = q < W ? bm[q] : 0u;
                    vvc += __popc(word);
                    int c = __popc(upper_bits(word, q, x));
                    int incl = warp_incl_scan(c, lane);
                    if (q < W) pre[q] = run + incl - c;
                    run += __shfl_sync(FULL, incl, 31);
                }
                ec = run;
                vvc = warp_sum(vvc);
                etv = warp_sum(etv);
                bad = ec > caps.max_up;
            }
            if (lane == 0) {
                scnt[3 * warp + 0] = active ? vvc : 0;
                scnt[3 * warp + 1] = active ? ec : 0;
                scnt[3 * warp + 2] = active ? etv : 0;
            }
            if (__syncthreads_or(bad && lane == 0)) {
                if (tid == 0) atomicOr(err, ERR_CAPACITY);
                return;
            }
            if (warp == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    int v = lane < NWARP ? scnt[3 * lane + c] : 0;
                    int incl = warp_incl_scan(v, lane);
                    int tot = __shfl_sync(FULL, incl, 31);
                    int cb = carry[c];
                    if (lane < NWARP) sbase[3 * lane + c] = cb + incl - v;
                    if (!COUNT && lane < NWARP && r0 + lane < nvo) {
                        if (c == 0 && (mask & R_VV)) it->vv_off[r0 + lane] = cb + incl - v;
                        if (c == 1 && (mask & R_ET)) it->eu_off[r0 + lane] = cb + incl - v;
                    }
                    __syncwarp();
                    if (lane == 0) carry[c] = cb + tot;
                }
            }
            __syncthreads();
            if (active && (do_vv || do_et)) {
                const int vbase = sbase[3 * warp + 0];
                const int ebase = sbase[3 * warp + 1];
                const int tbase = sbase[3 * warp + 2];
                // VV row and the upper endpoints of x's edges, in bit order
                int run_v = 0, run_e = 0;
                for (int q0 = 0; q0 < W; q0 += 32) {
                    const int q = q0 + lane;
                    uint32_t word = q < W ? bm[q] : 0u;
                    uint32_t up = upper_bits(word, q, x);
                    int cv = __popc(word), cu = __popc(up);
                    int iv = warp_incl_scan(cv, lane), iu = warp_incl_scan(cu, lane);
                    int pv = vbase + run_v + iv - cv, pu = ebase + run_e + iu - cu;
                    if (do_vv) {
                        uint32_t wv = word;
                        while (wv) {
                            int b = __ffs(wv) - 1;
                            wv &= wv - 1;
                            it->vv_val[pv++] = vmap[q * 32 + b];
                        }
                    }
                    if (do_et) {
                        uint32_t wu = up;
                        while (wu) {
                            int b = __ffs(wu) - 1;
                            wu &= wu - 1;
                            it->e_w[pu++] = vmap[q * 32 + b];
                        }
                    }
                    run_v += __shfl_sync(FULL, iv, 31);
                    run_e += __shfl_sync(FULL, iu, 31);
                }
                if (do_et) {
                    // ET rows of the edges (x, w): ranks from the bitmap prefix
                    const int E = ec;
                    auto rank = [&](uint32_t y) -> int {
                        int q = int(y >> 5);
                        uint32_t below = (y & 31) ? (FULL >> (32 - (y & 31))) : 0u;
                        return pre[q] + __popc(upper_bits(bm[q], q, x) & below);
                    };
                    const int nch = (L + 31) >> 5;
                    if (nch > 1) {
                        for (int e = lane; e < E; e += 32) ecnt[e] = 0;
                        __syncwarp();
                        for (int j = lane; j < L; j += 32) {
                            uint2 r = rows[S.vt_list[beg + j]];
#pragma unroll
                            for (int s = 0; s < 4; ++s) {
                                uint32_t y = vtx(r, s);
                                if (int(y) > x) atomicAdd(&ecnt[rank(y)], 1);
                            }
                        }
                        __syncwarp();
                        int run = 0;
                        for (int e0 = 0; e0 < E; e0 += 32) {
                            const int e = e0 + lane;
                            int c = e < E ? ecnt[e] : 0;
                            int incl = warp_incl_scan(c, lane);
                            if (e < E) {
                                ecnt[e] = run + incl - c;
                                it->et_off[ebase + e] = tbase + run + incl - c;
                            }
                            run += __shfl_sync(FULL, incl, 31);
                        }
                        __syncwarp();
                    }
                    for (int ch = 0; ch < nch; ++ch) {
                        for (int e = lane; e < E; e += 32) emask[e] = 0;
                        __syncwarp();
                        const int j = ch * 32 + lane;
                        uint2 r = make_uint2(0, 0);
                        int32_t tg = 0;
                        if (j < L) {
                            const int tl = S.vt_list[beg + j];
                            r = rows[tl];
                            tg = glob_tet(h, tmap, tl);
#pragma unroll
                            for (int s = 0; s < 4; ++s) {
                                uint32_t y = vtx(r, s);
                                if (int(y) > x) atomicOr(&emask[rank(y)], 1u << lane);
                            }
                        }
                        __syncwarp();
                        if (nch == 1) {
                            // single chunk: starts from the popcounts of the masks
                            int run = 0;
                            for (int e0 = 0; e0 < E; e0 += 32) {
                                const int e = e0 + lane;
                                int c = e < E ? __popc(emask[e]) : 0;
                                int incl = warp_incl_scan(c, lane);
                                if (e < E) {
                                    ecnt[e] = run + incl - c;
                                    it->et_off[ebase + e] = tbase + run + incl - c;
                                }
                                run += __shfl_sync(FULL, incl, 31);
                            }
                            __syncwarp();
                        }
                        if (j < L) {
                            const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
                            for (int s = 0; s < 4; ++s) {
                                uint32_t y = vtx(r, s);
                                if (int(y) > x) {
                                    int e = rank(y);
                                    it->et_val[tbase + ecnt[e] + __popc(emask[e] & lt)] = tg;
                                }
                            }
                        }
                        __syncwarp();
                        if (nch > 1) {
                            for (int e = lane; e < E; e += 32) ecnt[e] += __popc(emask[e]);
                            __syncwarp();
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            if (COUNT) {
                sizes_out[SZ_VV] = carry[0];
                sizes_out[SZ_E] = carry[1];
                sizes_out[SZ_ET] = carry[2];
            } else {
                if (mask & R_VV) it->vv_off[nvo] = carry[0];
                if (mask & R_ET) {
                    it->eu_off[nvo] = carry[1];
                    it->et_off[carry[1]] = carry[2];
                }
            }
        }
        __syncthreads();
    }

    if (COUNT || (mask & R_TT)) {
        // ---------------- D. TT ----------------
        const int n_own = h.n_own, n_ext = h.n_ext;
        const uint32_t hmask = uint32_t(caps.hcap - 1);
        uint32_t *hash = S.hash;
        uint32_t *nbr = S.nbr;  // neighbour across face s of internal tet i: nbr[4 i + s], ~0u = none
        for (int i = tid; i < caps.hcap; i += NT) hash[i] = 0u;
        for (int i = tid; i < 4 * n_own; i += NT) nbr[i] = 0xffffffffu;
        __syncthreads();
        int32_t flags = 0;
        for (int i = tid; i < n_own; i += NT) {
            const uint2 r = rows[n_ext + i];
            for (int s = 0; s < 4; ++s) {
                const uint64_t key = face_key(r, s);
                uint32_t hp = face_hash(key, hmask);
                int probe = 0;
                for (; probe < caps.hcap; ++probe) {
                    uint32_t prev = atomicCAS(&hash[hp], 0u, uint32_t(i * 4 + s + 1));
                    if (prev == 0u) break;
                    const uint32_t ref = prev - 1u;
                    const int i2 = int(ref >> 2), s2 = int(ref & 3u);
                    if (face_key(rows[n_ext + i2], s2) == key) {
                        const uint32_t o1 = atomicCAS(&nbr[i2 * 4 + s2], 0xffffffffu, uint32_t(n_ext + i));
                        const uint32_t o2 = atomicCAS(&nbr[i * 4 + s], 0xffffffffu, uint32_t(n_ext + i2));
                        if (o1 != 0xffffffffu || o2 != 0xffffffffu) flags |= ERR_NONMANIFOLD;
                        break;
                    }
                    hp = (hp + 1u) & hmask;
                }
                if (probe == caps.hcap) flags |= ERR_HASH_FULL;
            }
        }
        __syncthreads();
        const int nprobe = n_ext + h.n_halo;
        for (int j = tid; j < nprobe; j += NT) {
            const int tl = j < n_ext ? j : n_own + j;
            const uint2 r = rows[tl];
            for (int s = 0; s < 4; ++s) {
                const uint64_t key = face_key(r, s);
                uint32_t hp = face_hash(key, hmask);
                for (int probe = 0; probe < caps.hcap; ++probe) {
                    const uint32_t e = hash[hp];
                    if (e == 0u) break;
                    const uint32_t ref = e - 1u;
                    const int i2 = int(ref >> 2), s2 = int(ref & 3u);
                    if (face_key(rows[n_ext + i2], s2) == key) {
                        const uint32_t o = atomicCAS(&nbr[i2 * 4 + s2], 0xffffffffu, uint32_t(tl));
                        if (o != 0xffffffffu) flags |= ERR_NONMANIFOLD;
                        break;
                    }
                    hp = (hp + 1u) & hmask;
                }
            }
        }
        if (flags) atomicOr(err, flags);
        __syncthreads();
        int carry = 0;
        const bool do_tt = !COUNT && (mask & R_TT);
        for (int r0 = 0; r0 < n_own; r0 += NT) {
            const int i = r0 + tid;
            // absent neighbours sort last as INT32_MAX
            int32_t v0 = INT32_MAX, v1 = INT32_MAX, v2 = INT32_MAX, v3 = INT32_MAX;
            int c = 0;
            if (i < n_own) {
                const uint4 nb = *reinterpret_cast<const uint4 *>(&nbr[i * 4]);
                if (nb.x != 0xffffffffu) { v0 = glob_tet(h, tmap, int32_t(nb.x)); ++c; }
                if (nb.y != 0xffffffffu) { v1 = glob_tet(h, tmap, int32_t(nb.y)); ++c; }
                if (nb.z != 0xffffffffu) { v2 = glob_tet(h, tmap, int32_t(nb.z)); ++c; }
                if (nb.w != 0xffffffffu) { v3 = glob_tet(h, tmap, int32_t(nb.w)); ++c; }
                sort4_net(v0, v1, v2, v3);
            }
            int tot;
            const int pos = carry + block_scan_thread<NT>(c, S.scan, &tot);
            if (do_tt && i < n_own) {
                it->tt_off[i] = pos;
                int32_t *o = it->tt_val + pos;
                if (c > 0) o[0] = v0;
                if (c > 1) o[1] = v1;
                if (c > 2) o[2] = v2;
                if (c > 3) o[3] = v3;
            }
            carry += tot;
            __syncthreads();
        }
        if (tid == 0) {
            if (COUNT) sizes_out[SZ_TT] = carry;
            else if (do_tt) it->tt_off[n_own] = carry;
        }
    }
    __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT) count_kernel(DevMesh m, SmemPlan plan, const int32_t *ids, int32_t n,
                                                   int64_t *sizes, int32_t *err, int32_t *ticket) {
    extern __shared__ __align__(16) char smem[];
    const Smem S = carve(smem, plan);
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
        run_cluster<NT, true>(m, plan, S, m.blk_off[k], 0u, nullptr, s_sizes, err);
        __syncthreads();
        if (threadIdx.x < SZ_N) sizes[int64_t(k) * SZ_N + threadIdx.x] = s_sizes[threadIdx.x];
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) build_kernel(DevMesh m, SmemPlan plan, const WorkItem *items,
                                                   const int32_t *order, int32_t n, int32_t *err,
                                                   int32_t *ticket) {
    extern __shared__ __align__(16) char smem[];
    const Smem S = carve(smem, plan);
    __shared__ int32_t s_idx;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(ticket, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= n) break;
        const WorkItem *it = items + (order ? order[idx] : idx);
        const int k = it->k;
        if (k < 0 || k >= m.K) {
            if (threadIdx.x == 0) atomicOr(err, ERR_BAD_ITEM);
            continue;
        }
        run_cluster<NT, false>(m, plan, S, it->blk, it->mask, it, nullptr, err);
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) build_one_kernel(DevMesh m, SmemPlan plan, const WorkItem *items,
                                                       int32_t index, int32_t *err) {
    extern __shared__ __align__(16) char smem[];
    const Smem S = carve(smem, plan);
    const WorkItem *it = items + index;
    if (it->k < 0 || it->k >= m.K) {
        if (threadIdx.x == 0) atomicOr(err, ERR_BAD_ITEM);
        return;
    }
    run_cluster<NT, false>(m, plan, S, it->blk, it->mask, it, nullptr, err);
}

// Output placement (a5): exclusive scans, over the listed clusters, of every
// output array's length; one CTA.  arrays_base holds the base pointers of the
// ten bulk arrays (its k/mask/blk fields are ignored).
constexpr int kBasesThreads = 1024;
__global__ void __launch_bounds__(kBasesThreads) bases_kernel(DevMesh m, const int32_t *ids, int32_t n,
                                                              const int64_t *sizes, uint32_t mask,
                                                              const WorkItem *arrays_base, WorkItem *items,
                                                              int64_t *totals) {
    // per item lengths of the ten arrays
    constexpr int NA = 10;
    __shared__ int64_t s_warp[kBasesThreads / 32][NA];
    __shared__ int64_t s_tot[NA];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + kBasesThreads - 1) / kBasesThreads;
    const int b = tid * per, e = min(n, b + per);
    auto lens = [&](int idx, int64_t *L) {
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
    };
    int64_t acc[NA];
    for (int a = 0; a < NA; ++a) acc[a] = 0;
    for (int i = b; i < e; ++i) {
        int64_t L[NA];
        lens(i, L);
        for (int a = 0; a < NA; ++a) acc[a] += L[a];
    }
    // block exclusive scan of acc[]
    int64_t incl[NA];
    for (int a = 0; a < NA; ++a) {
        int64_t v = acc[a];
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += y;
        }
        incl[a] = v;
        if (lane == 31) s_warp[warp][a] = v;
    }
    __syncthreads();
    if (warp == 0) {
        for (int a = 0; a < NA; ++a) {
            int64_t w = s_warp[lane][a];
            int64_t v = w;
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(FULL, v, o);
                if (lane >= o) v += y;
            }
            s_warp[lane][a] = v - w;
            if (lane == 31) s_tot[a] = v;
        }
    }
    __syncthreads();
    int64_t run[NA];
    for (int a = 0; a < NA; ++a) run[a] = s_warp[warp][a] + incl[a] - acc[a];
    int32_t *base[NA] = {arrays_base->vt_off, arrays_base->vt_val, arrays_base->vv_off, arrays_base->vv_val,
                         arrays_base->eu_off, arrays_base->e_w, arrays_base->et_off, arrays_base->et_val,
                         arrays_base->tt_off, arrays_base->tt_val};
    for (int i = b; i < e; ++i) {
        int64_t L[NA];
        lens(i, L);
        const int k = ids ? ids[i] : i;
        WorkItem w;
        w.k = k;
        w.mask = mask;
        w.blk = m.blk_off[k];
        int32_t *p[NA];
        for (int a = 0; a < NA; ++a) p[a] = base[a] ? base[a] + run[a] : nullptr;
        w.vt_off = p[0]; w.vt_val = p[1]; w.vv_off = p[2]; w.vv_val = p[3];
        w.eu_off = p[4]; w.e_w = p[5]; w.et_off = p[6]; w.et_val = p[7];
        w.tt_off = p[8]; w.tt_val = p[9];
        items[i] = w;
        for (int a = 0; a < NA; ++a) run[a] += L[a];
    }
    if (tid < NA) totals[tid] = s_tot[tid];
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
    const int Wc = (c.nv_loc + 31) / 32;
    int64_t off = 0;
    p.blk = 0;
    off = a16(int64_t(4) * c.blk_words);
    p.scan = int32_t(off);
    off = a16(off + 4 * ((nwarp + 1) + 6 * nwarp + 3 + 8));
    p.vt_off = int32_t(off);
    off = a16(off + 4 * (int64_t(c.nv_own) + 1));
    p.cur = int32_t(off);
    off = a16(off + 4 * int64_t(c.nv_own));
    p.vt_list = int32_t(off);
    off = a16(off + 2 * int64_t(c.n_vt));
    p.uni = int32_t(off);
    p.warp_words = int32_t(((2 * Wc + 2 * c.max_up) + 3) & ~3);
    const int64_t uni_b = 4 * int64_t(nwarp) * c.nv_own;
    const int64_t uni_c = 4 * int64_t(nwarp) * p.warp_words;
    const int64_t end_bc = a16(off + (uni_b > uni_c ? uni_b : uni_c));
    p.hash = p.vt_off;
    p.nbr = int32_t(a16(int64_t(p.hash) + 4 * int64_t(c.hcap)));
    const int64_t end_d = a16(int64_t(p.nbr) + 16 * int64_t(c.n_own));
    p.total = int32_t(end_bc > end_d ? end_bc : end_d);
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

template <int NT>
static const void *build_fn() { return reinterpret_cast<const void *>(&build_kernel<NT>); }

int max_ctas_per_sm(const SmemPlan &plan) {
    int n = 0;
    const void *fn = plan.threads == 128 ? build_fn<128>() : plan.threads == 256 ? build_fn<256>() : build_fn<512>();
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.total);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, plan.threads, plan.total) != cudaSuccess) return 0;
    return n;
}

template <class F>
static int dispatch_threads(int nt, F &&f) {
    switch (nt) {
        case 128: f(std::integral_constant<int, 128>{}); break;
        case 256: f(std::integral_constant<int, 256>{}); break;
        case 512: f(std::integral_constant<int, 512>{}); break;
        default: return int(cudaErrorInvalidValue);
    }
    return int(cudaGetLastError());
}

int launch_count_pass(const DevMesh &m, const SmemPlan &plan, const int32_t *ids, int32_t n, int64_t *sizes_out,
                      int32_t *err, int32_t *ticket, int grid, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(ticket, 0, sizeof(int32_t), s);
    return dispatch_threads(plan.threads, [&](auto ntc) {
        constexpr int NT = decltype(ntc)::value;
        cudaFuncSetAttribute(count_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.total);
        count_kernel<NT><<<grid, NT, plan.total, s>>>(m, plan, ids, n, sizes_out, err, ticket);
    });
}

int launch_bases(const DevMesh &m, const int32_t *ids, int32_t n, const int64_t *sizes, uint32_t mask,
                 const WorkItem *arrays_base, WorkItem *items, int64_t *totals_out, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bases_kernel<<<1, kBasesThreads, 0, s>>>(m, ids, n, sizes, mask, arrays_base, items, totals_out);
    return int(cudaGetLastError());
}

int launch_build(const DevMesh &m, const SmemPlan &plan, const WorkItem *items, const int32_t *order, int32_t n,
                 int32_t *err, int32_t *ticket, int grid, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(ticket, 0, sizeof(int32_t), s);
    return dispatch_threads(plan.threads, [&](auto ntc) {
        constexpr int NT = decltype(ntc)::value;
        build_kernel<NT><<<grid, NT, plan.total, s>>>(m, plan, items, order, n, err, ticket);
    });
}

int launch_build_one(const DevMesh &m, const SmemPlan &plan, const WorkItem *items, int32_t index, int32_t *err,
                     void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return dispatch_threads(plan.threads, [&](auto ntc) {
        constexpr int NT = decltype(ntc)::value;
        build_one_kernel<NT><<<1, NT, plan.total, s>>>(m, plan, items, index, err);
    });
}

void prepare_kernels(int threads, int smem) {
    dispatch_threads(threads, [&](auto ntc) {
        constexpr int NT = decltype(ntc)::value;
        cudaFuncSetAttribute(build_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(build_one_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
}

}  // namespace gale
