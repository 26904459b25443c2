// Coboundary relations VE, VF, EF, FT in the ids of the edge / triangle
// enumeration (Section 4.4: coboundary relations are computed by the GPU for
// whole segments; Section 5 evaluates VE, VF, EF and FT among them).
//
// Inputs on the device: the canonical tet rows, each vertex's cluster, the
// enumeration (E, F, I_E, I_F and each segment's ids in vertex-tuple order)
// and the VT, VV and ET rows of every cluster from a batched build.
//
// Lookup structure, built once per enumeration: the edges and triangles in
// vertex-tuple ("sorted") order, with
//   eo[v]    first sorted edge position with lower vertex v (nv+1 entries),
//   ekw[j]   upper vertex of the j-th sorted edge,
//   feo[j]   first sorted triangle position whose first two vertices are the
//            j-th sorted edge (nE+1 entries),
//   fkc[p]   third vertex of the p-th sorted triangle,
//   e2s, f2s the sorted position of every edge / triangle id.
// An edge (a, b) is then found among a's few upper edges and a triangle
// (a, b, c) among the few triangles over its edge (a, b).  Within a segment
// the sorted edge order is the order of the cluster's ET rows (own lower
// vertex, then upper vertex), so the tets around the j-th sorted edge are
// the ET row at j - I_E[k] of its cluster k.
//
// One thread per output row, two passes (count, then fill after an
// exclusive scan):
//   VE(v)  the edges {v, w} for w in VV(v);
//   EF(e)  the triangles (u, w, x) for the distinct third vertices x of the
//          tets of ET(e);
//   VF(v)  read from EF: a triangle through v has two edges through v, and
//          is taken from the one to its smaller other vertex (so EF is built
//          first, and whenever VF is asked for);
//   FT(f)  for f = (a, b, c): the tets of ET(a, b) that contain c.
// With the sorted numbering every row comes out ascending; otherwise rows
// whose ids come from lookups are sorted in place.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gale_ctx.h"
#include "gale_enum.h"

namespace gale {

// device copies the coboundary pass keeps in the context
struct Cobound {
    uint64_t enm_gen = 0;  // the enumeration the lookup index was made from
    uint64_t dev_gen = 0;  // the enumeration E, F, IE, IF (and ebk, fbk) hold
    int32_t *rows = nullptr, *cluster_of = nullptr;
    int32_t *E = nullptr, *F = nullptr, *ebk = nullptr, *fbk = nullptr;
    int64_t *IE = nullptr, *IF = nullptr;
    int32_t *eo = nullptr, *ekw = nullptr, *feo = nullptr, *fkc = nullptr, *fo = nullptr;
    int32_t *e2s = nullptr, *f2s = nullptr;
    bool sorted_ids = false;
    int64_t *base = nullptr;       // [K][10] bulk bases of every cluster's arrays
    int32_t *cnt = nullptr;        // counts of the largest relation
    int64_t *bsum = nullptr;       // scan block sums
    int64_t cnt_cap = 0, bsum_cap = 0;
    int32_t *off[4] = {}, *val[4] = {};
    int32_t *ef_third = nullptr;   // per EF entry: the triangle's vertex off the edge
    int64_t ef_third_cap = 0;
    int64_t off_cap[4] = {}, val_cap[4] = {};
    int64_t rows_of[4] = {}, len[4] = {};
};

void cobound_destroy(gale_ctx *ctx) {
    delete ctx->cb;  // device memory is the context's and goes with it
    ctx->cb = nullptr;
}

namespace {

constexpr int kThreads = 256;
enum { REL_VE = 0, REL_VF = 1, REL_EF = 2, REL_FT = 3 };
// bulk array indices (the order of gale_arrays)
enum { B_VT_OFF = 0, B_VT_VAL = 1, B_VV_OFF = 2, B_VV_VAL = 3, B_ET_UOFF = 4, B_ET_W = 5, B_ET_OFF = 6, B_ET_VAL = 7 };

struct CbMesh {
    const int4 *rows;
    const int32_t *cluster_of, *I_V;
    const int32_t *E, *F, *ebk, *fbk;
    const int64_t *IE, *IF;
    const int32_t *eo, *ekw, *feo, *fkc, *e2s, *f2s;
    const int32_t *vt_off, *vt_val, *vv_off, *vv_val, *et_w, *et_off, *et_val;
    const int32_t *et_uoff;          // ET edges per own lower vertex (the sorted enumeration reads it)
    const int32_t *ef_off, *ef_val;  // EF, once built (VF is read from it)
    const int32_t *ve_off, *ve_val;  // VE in VV order, once built (VF is read from it)
    const int32_t *ef_third;         // per EF entry: the triangle's vertex off the edge
    int32_t *third_out;              // where the EF fill writes those
    const int64_t *base;
    const int64_t *sizes;  // [K][5] per-cluster entries: VT, VV, edges, ET, TT
    int64_t nv, nE, nF;
    bool sorted_ids;
};

// [b, e) of vertex v's row of a per-own-vertex bulk relation (VT or VV)
__device__ __forceinline__ void vrow(const CbMesh &m, int32_t v, bool vv, int64_t &b, int64_t &e) {
    const int32_t k = m.cluster_of[v];
    const int32_t i = v - m.I_V[k];
    const int32_t *off = vv ? m.vv_off : m.vt_off;
    const int64_t *B = m.base + 10 * int64_t(k);
    const int64_t ob = B[vv ? B_VV_OFF : B_VT_OFF], vb = B[vv ? B_VV_VAL : B_VT_VAL];
    b = vb + off[ob + i];
    e = vb + off[ob + i + 1];
}

__device__ __forceinline__ bool has4(const int4 r, int32_t x) { return r.x == x || r.y == x || r.z == x || r.w == x; }

// sorted position of edge (a, b), a < b, or -1
__device__ int64_t epos(const CbMesh &m, int32_t a, int32_t b) {
    int64_t lo = m.eo[a];
    const int64_t end = m.eo[a + 1];
    int64_t hi = end;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (m.ekw[mid] < b) lo = mid + 1;
        else hi = mid;
    }
    return (lo < end && m.ekw[lo] == b) ? lo : -1;
}

// sorted position of triangle (a, b, c), a < b < c, whose edge (a, b) has
// sorted position j, or -1
__device__ int64_t fpos_at(const CbMesh &m, int64_t j, int32_t c) {
    const int64_t end = m.feo[j + 1];
    for (int64_t p = m.feo[j]; p < end; ++p) {
        const int32_t x = m.fkc[p];
        if (x == c) return p;
        if (x > c) break;
    }
    return -1;
}

// sorted position of triangle (a, b, c), a < b < c, or -1
__device__ int64_t fpos(const CbMesh &m, int32_t a, int32_t b, int32_t c) {
    const int64_t j = epos(m, a, b);
    return j < 0 ? -1 : fpos_at(m, j, c);
}

__device__ __forceinline__ void sort3(int32_t &a, int32_t &b, int32_t &c) {
    if (a > b) { const int32_t t = a; a = b; b = t; }
    if (b > c) { const int32_t t = b; b = c; c = t; }
    if (a > b) { const int32_t t = a; a = b; b = t; }
}

// the ET row [b, e) of the edge at sorted position j, whose vertices are
// (a, w); false if the cluster's ET rows do not list that edge there
__device__ bool et_row(const CbMesh &m, int64_t j, int32_t a, int32_t w, int64_t &b, int64_t &e) {
    const int32_t k = m.cluster_of[a];
    const int64_t le = j - m.IE[k];
    if (le < 0 || j >= m.IE[k + 1] || le >= m.sizes[5 * int64_t(k) + 2]) return false;
    const int64_t *B = m.base + 10 * int64_t(k);
    if (m.et_w[B[B_ET_W] + le] != w) return false;
    b = B[B_ET_VAL] + m.et_off[B[B_ET_OFF] + le];
    e = B[B_ET_VAL] + m.et_off[B[B_ET_OFF] + le + 1];
    return true;
}

__device__ __forceinline__ int32_t edge_id(const CbMesh &m, int64_t j) { return m.sorted_ids ? int32_t(j) : m.ebk[j]; }
__device__ __forceinline__ int32_t face_id(const CbMesh &m, int64_t p) { return m.sorted_ids ? int32_t(p) : m.fbk[p]; }

// One row of relation REL: count (out == nullptr) or write its entries (at
// most cap of them; the count is returned either way).
template <int REL>
__device__ int32_t row_entries(const CbMesh &m, int64_t row, int32_t *out, int32_t cap, int32_t *aux,
                               int32_t *err) {
    int32_t n = 0;
    if (REL == REL_VE) {
        const int32_t v = int32_t(row);
        int64_t b, e;
        vrow(m, v, true, b, e);
        if (!out) return int32_t(e - b);
        for (int64_t j = b; j < e; ++j) {
            const int32_t w = m.vv_val[j];
            const int64_t p = v < w ? epos(m, v, w) : epos(m, w, v);
            if (p < 0) atomicOr(err, ERR_BAD_BLOCK);
            if (n < cap) out[n] = p < 0 ? -1 : edge_id(m, p);
            ++n;
        }
    } else if (REL == REL_VF) {
        // every triangle through v has exactly two edges through v: take it
        // from the one to its smaller other vertex.  With x ascending and
        // EF rows ordered by third vertex, the sorted numbering's ids come
        // out ascending.
        // VE(v) is still in VV(v)'s order here: entry i is the edge to the
        // i-th neighbour
        const int32_t v = int32_t(row);
        int64_t b, e;
        vrow(m, v, true, b, e);
        const int64_t vb = m.ve_off[v];
        if (m.ve_off[v + 1] - vb != e - b) {
            atomicOr(err, ERR_BAD_BLOCK);
            return 0;
        }
        for (int64_t j = b; j < e; ++j) {
            const int32_t x = m.vv_val[j];
            const int32_t id = m.ve_val[vb + (j - b)];
            if (id < 0) {
                atomicOr(err, ERR_BAD_BLOCK);
                return n;
            }
            const int32_t fb = m.ef_off[id], fe = m.ef_off[id + 1];
            if (!out) {
                n += fe - fb;  // halved below: each triangle is met twice
                continue;
            }
            for (int32_t q = fb; q < fe; ++q)
                if (m.ef_third[q] > x) {
                    if (n < cap) out[n] = m.ef_val[q];
                    ++n;
                }
        }
        if (!out) n >>= 1;
    } else if (REL == REL_EF) {
        // the third vertices of the tets around e, sorted and deduplicated:
        // with the sorted numbering, ascending third vertex is ascending id
        const int64_t js = m.sorted_ids ? row : m.e2s[row];
        const int32_t u = m.E[2 * row], w = m.E[2 * row + 1];
        int64_t eb, ee;
        if (!et_row(m, js, u, w, eb, ee)) {
            atomicOr(err, ERR_BAD_BLOCK);
            return 0;
        }
        constexpr int kCand = 32;
        if (ee - eb <= kCand / 2) {
            int32_t xs[kCand];
            int c = 0;
            for (int64_t j = eb; j < ee; ++j) {
                const int4 r = m.rows[m.et_val[j]];
#pragma unroll
                for (int s2 = 0; s2 < 4; ++s2) {
                    const int32_t x = s2 == 0 ? r.x : s2 == 1 ? r.y : s2 == 2 ? r.z : r.w;
                    if (x == u || x == w || c >= kCand) continue;
                    int q = c++;
                    while (q > 0 && xs[q - 1] > x) {
                        xs[q] = xs[q - 1];
                        --q;
                    }
                    xs[q] = x;
                }
            }
            for (int q = 0; q < c; ++q) {
                if (q > 0 && xs[q] == xs[q - 1]) continue;
                if (out && n < cap) {
                    const int32_t x = xs[q];
                    int64_t p;
                    if (x > w) {
                        p = fpos_at(m, js, x);  // (u, w, x): over this edge
                    } else {
                        int32_t a = u, bb = w, cc = x;
                        sort3(a, bb, cc);
                        p = fpos(m, a, bb, cc);
                    }
                    if (p < 0) atomicOr(err, ERR_BAD_BLOCK);
                    out[n] = p < 0 ? -1 : face_id(m, p);
                    if (aux) aux[n] = x;
                }
                ++n;
            }
            return n;
        }
        // many tets around the edge: first-occurrence test over the row
        for (int64_t j = eb; j < ee; ++j) {
            const int4 r = m.rows[m.et_val[j]];
#pragma unroll
            for (int s2 = 0; s2 < 4; ++s2) {
                const int32_t x = s2 == 0 ? r.x : s2 == 1 ? r.y : s2 == 2 ? r.z : r.w;
                if (x == u || x == w) continue;
                bool first = true;
                for (int64_t jj = eb; jj < j && first; ++jj) first = !has4(m.rows[m.et_val[jj]], x);
                if (!first) continue;
                if (out && n < cap) {
                    int32_t a = u, bb = w, cc = x;
                    sort3(a, bb, cc);
                    const int64_t p = fpos(m, a, bb, cc);
                    if (p < 0) atomicOr(err, ERR_BAD_BLOCK);
                    out[n] = p < 0 ? -1 : face_id(m, p);
                    if (aux) aux[n] = x;
                }
                ++n;
            }
        }
    } else {
        const int32_t a = m.F[3 * row], bb = m.F[3 * row + 1], cc = m.F[3 * row + 2];
        const int64_t je = epos(m, a, bb);
        int64_t eb, ee;
        if (je < 0 || !et_row(m, je, a, bb, eb, ee)) {
            atomicOr(err, ERR_BAD_BLOCK);
            return 0;
        }
        for (int64_t j = eb; j < ee; ++j) {
            const int32_t t = m.et_val[j];
            if (has4(m.rows[t], cc)) {
                if (out && n < cap) out[n] = t;
                ++n;
            }
        }
    }
    return n;
}

template <int REL>
__global__ void __launch_bounds__(kThreads) cb_count(CbMesh m, int64_t rows, int32_t *cnt, int32_t *err) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x)
        cnt[r] = row_entries<REL>(m, r, nullptr, 0, nullptr, err);
}

template <int REL>
__global__ void __launch_bounds__(kThreads) cb_fill(CbMesh m, int64_t rows, const int32_t *off, int32_t *val,
                                                    int32_t *err) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x) {
        int32_t *o = val + off[r];
        const int32_t len = off[r + 1] - off[r];
        int32_t *ax = REL == REL_EF ? m.third_out + off[r] : nullptr;
        const int32_t n = row_entries<REL>(m, r, o, len, ax, err);
        if (n != len) {
            atomicOr(err, ERR_BAD_BLOCK);
            continue;
        }
        // VE stays in VV order until VF has read it (cb_sort_rows sorts it)
        const bool need_sort = REL == REL_VF || REL == REL_EF;
        if (need_sort)  // ids found by lookup: sort the row (insertion sort)
            for (int32_t i = 1; i < n; ++i) {
                const int32_t x = o[i];
                const int32_t y = ax ? ax[i] : 0;
                int32_t j = i - 1;
                while (j >= 0 && o[j] > x) {
                    o[j + 1] = o[j];
                    if (ax) ax[j + 1] = ax[j];
                    --j;
                }
                o[j + 1] = x;
                if (ax) ax[j + 1] = y;
            }
    }
}

// sort every row of a CSR relation in place (insertion sort; rows are short)
__global__ void __launch_bounds__(kThreads) cb_sort_rows(int64_t rows, const int32_t *off, int32_t *val) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x) {
        int32_t *o = val + off[r];
        const int32_t n = off[r + 1] - off[r];
        for (int32_t i = 1; i < n; ++i) {
            const int32_t x = o[i];
            int32_t j = i - 1;
            while (j >= 0 && o[j] > x) {
                o[j + 1] = o[j];
                --j;
            }
            o[j + 1] = x;
        }
    }
}

// ---- sorted enumeration on the device ----
// A segment's edges in vertex-tuple order are its cluster's ET edges (own
// lower vertex u, then upper vertex w): E is written straight from the ET
// rows.  Its triangles over an edge (a, b) are (a, b, c) for the distinct
// vertices c > b of the tets of ET(a, b), ascending.

// E pairs of every cluster's edges, at I_E[k] + local edge index
__global__ void __launch_bounds__(kThreads) k_enum_edges(CbMesh m, int32_t *E) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < m.nv; v += int64_t(gridDim.x) * blockDim.x) {
        const int32_t k = m.cluster_of[v];
        const int32_t i = int32_t(v) - m.I_V[k];
        const int64_t *B = m.base + 10 * int64_t(k);
        const int32_t e0 = m.et_uoff[B[B_ET_UOFF] + i], e1 = m.et_uoff[B[B_ET_UOFF] + i + 1];
        for (int32_t e = e0; e < e1; ++e) {
            const int64_t j = m.IE[k] + e;
            E[2 * j] = int32_t(v);
            E[2 * j + 1] = m.et_w[B[B_ET_W] + e];
        }
    }
}

// triangles over each edge: count (F == nullptr) or write at FS[j]
template <bool WRITE>
__global__ void __launch_bounds__(kThreads) k_enum_faces(CbMesh m, const int32_t *E, int32_t *nf, const int32_t *FS,
                                                         int32_t *F, int32_t *err) {
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < m.nE; j += int64_t(gridDim.x) * blockDim.x) {
        const int32_t a = E[2 * j], b = E[2 * j + 1];
        int64_t eb, ee;
        if (!et_row(m, j, a, b, eb, ee)) {
            atomicOr(err, ERR_BAD_BLOCK);
            if (!WRITE) nf[j] = 0;
            continue;
        }
        int32_t n = 0;
        int64_t out = WRITE ? FS[j] : 0;
        const int64_t cap = WRITE ? FS[j + 1] - FS[j] : 0;
        constexpr int kCand = 32;
        if (ee - eb <= kCand / 2) {
            int32_t xs[kCand];
            int c = 0;
            for (int64_t q = eb; q < ee; ++q) {
                const int4 r = m.rows[m.et_val[q]];
#pragma unroll
                for (int s2 = 0; s2 < 4; ++s2) {
                    const int32_t x = s2 == 0 ? r.x : s2 == 1 ? r.y : s2 == 2 ? r.z : r.w;
                    if (x <= b || c >= kCand) continue;
                    int p = c++;
                    while (p > 0 && xs[p - 1] > x) {
                        xs[p] = xs[p - 1];
                        --p;
                    }
                    xs[p] = x;
                }
            }
            for (int p = 0; p < c; ++p) {
                if (p > 0 && xs[p] == xs[p - 1]) continue;
                if (WRITE && n < cap) {
                    F[3 * (out + n)] = a;
                    F[3 * (out + n) + 1] = b;
                    F[3 * (out + n) + 2] = xs[p];
                }
                ++n;
            }
        } else {
            // many tets around the edge: emit each c once, in increasing order
            int32_t last = b;
            for (;;) {
                int32_t next = INT32_MAX;
                for (int64_t q = eb; q < ee; ++q) {
                    const int4 r = m.rows[m.et_val[q]];
                    const int32_t xv[4] = {r.x, r.y, r.z, r.w};
                    for (int s2 = 0; s2 < 4; ++s2)
                        if (xv[s2] > last && xv[s2] < next) next = xv[s2];
                }
                if (next == INT32_MAX) break;
                if (WRITE && n < cap) {
                    F[3 * (out + n)] = a;
                    F[3 * (out + n) + 1] = b;
                    F[3 * (out + n) + 2] = next;
                }
                ++n;
                last = next;
            }
        }
        if (!WRITE) nf[j] = n;
        else if (n != cap) atomicOr(err, ERR_BAD_BLOCK);
    }
}

// I_F[k] = FS[I_E[k]] for k = 0..K
__global__ void __launch_bounds__(kThreads) k_enum_if(const int64_t *IE, const int32_t *FS, int64_t K, int64_t *IF) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k <= K; k += int64_t(gridDim.x) * blockDim.x)
        IF[k] = FS[IE[k]];
}

// ---- lookup structure, once per enumeration ----

// eo[v]: first sorted edge position of lower vertex v within its segment
__global__ void __launch_bounds__(kThreads) k_eo(CbMesh m, int32_t *eo) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v <= m.nv; v += int64_t(gridDim.x) * blockDim.x) {
        if (v == m.nv) {
            eo[v] = int32_t(m.nE);
            continue;
        }
        const int32_t k = m.cluster_of[v];
        int64_t lo = m.IE[k], hi = m.IE[k + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (m.E[2 * int64_t(edge_id(m, mid))] < v) lo = mid + 1;
            else hi = mid;
        }
        eo[v] = int32_t(lo);
    }
}

// fo[v]: first sorted triangle position of lowest vertex v
__global__ void __launch_bounds__(kThreads) k_fo(CbMesh m, int32_t *fo) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v <= m.nv; v += int64_t(gridDim.x) * blockDim.x) {
        if (v == m.nv) {
            fo[v] = int32_t(m.nF);
            continue;
        }
        const int32_t k = m.cluster_of[v];
        int64_t lo = m.IF[k], hi = m.IF[k + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (m.F[3 * int64_t(face_id(m, mid))] < v) lo = mid + 1;
            else hi = mid;
        }
        fo[v] = int32_t(lo);
    }
}

// ekw and e2s over sorted edge positions; fkc and f2s over triangle positions
__global__ void __launch_bounds__(kThreads) k_keys(CbMesh m, int32_t *ekw, int32_t *e2s, int32_t *fkc,
                                                   int32_t *f2s) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < m.nE; j += stride) {
        const int32_t id = edge_id(m, j);
        ekw[j] = m.E[2 * int64_t(id) + 1];
        e2s[id] = int32_t(j);
    }
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < m.nF; p += stride) {
        const int32_t id = face_id(m, p);
        fkc[p] = m.F[3 * int64_t(id) + 2];
        f2s[id] = int32_t(p);
    }
}

// feo[j]: first sorted triangle position over the j-th sorted edge (a, b)
__global__ void __launch_bounds__(kThreads) k_feo(CbMesh m, const int32_t *fo, int32_t *feo) {
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j <= m.nE; j += int64_t(gridDim.x) * blockDim.x) {
        if (j == m.nE) {
            feo[j] = int32_t(m.nF);
            continue;
        }
        const int32_t id = edge_id(m, j);
        const int32_t a = m.E[2 * int64_t(id)], b = m.E[2 * int64_t(id) + 1];
        int64_t lo = fo[a], hi = fo[a + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (m.F[3 * int64_t(face_id(m, mid)) + 1] < b) lo = mid + 1;
            else hi = mid;
        }
        feo[j] = int32_t(lo);
    }
}

// exclusive scan of cnt[0..n) into off[0..n]: block sums, one pass over the
// block sums, then the per-block scans
__global__ void __launch_bounds__(kThreads) scan_sums(const int32_t *cnt, int64_t n, int64_t *bsum) {
    __shared__ int64_t s[kThreads];
    const int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    s[threadIdx.x] = i < n ? cnt[i] : 0;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}

// exclusive scan of the nb block sums in place (bsum[nb] = total), one
// block: each thread sums a contiguous chunk, the chunk totals are scanned,
// then each thread rewrites its chunk
__global__ void __launch_bounds__(kThreads) scan_bsums(int64_t *bsum, int64_t nb) {
    __shared__ int64_t s[kThreads];
    const int64_t per = (nb + kThreads - 1) / kThreads;
    const int64_t b0 = min(nb, int64_t(threadIdx.x) * per), b1 = min(nb, b0 + per);
    int64_t sum = 0;
    for (int64_t b = b0; b < b1; ++b) sum += bsum[b];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < kThreads; o <<= 1) {
        const int64_t y = int(threadIdx.x) >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += y;
        __syncthreads();
    }
    int64_t run = s[threadIdx.x] - sum;
    for (int64_t b = b0; b < b1; ++b) {
        const int64_t x = bsum[b];
        bsum[b] = run;
        run += x;
    }
    if (threadIdx.x == kThreads - 1) bsum[nb] = s[kThreads - 1];
}

__global__ void __launch_bounds__(kThreads) scan_write(const int32_t *cnt, int64_t n, const int64_t *bsum,
                                                       int32_t *off, int64_t nb, int32_t *err) {
    __shared__ int64_t s[kThreads];
    const int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    const int64_t x = i < n ? cnt[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < kThreads; o <<= 1) {
        const int64_t y = int(threadIdx.x) >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += y;
        __syncthreads();
    }
    const int64_t ex = bsum[blockIdx.x] + s[threadIdx.x] - x;
    if (ex > INT32_MAX) atomicOr(err, ERR_CAPACITY);
    if (i < n) off[i] = int32_t(ex);
    if (i == 0) {
        const int64_t tot = bsum[nb];
        if (tot > INT32_MAX) atomicOr(err, ERR_CAPACITY);
        off[n] = int32_t(tot);
    }
}

gale_status fail(gale_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

template <class T>
bool grow(gale_ctx *ctx, T *&p, int64_t &cap, int64_t need) {
    if (need <= cap && p) return true;
    if (p) ctx->dfree(p);
    p = nullptr;
    cap = 0;
    const int64_t c = std::max<int64_t>(need + need / 8, 64);
    p = static_cast<T *>(ctx->dalloc(size_t(c) * sizeof(T)));
    if (!p) return false;
    cap = c;
    return true;
}

template <class T>
T *upload(gale_ctx *ctx, const T *h, size_t n, cudaStream_t s) {
    T *d = static_cast<T *>(ctx->dalloc(std::max<size_t>(n, 1) * sizeof(T)));
    if (d && n) cudaMemcpyAsync(d, h, n * sizeof(T), cudaMemcpyHostToDevice, s);
    return d;
}
template <class T>
T *upload(gale_ctx *ctx, const std::vector<T> &h, cudaStream_t s) {
    return upload(ctx, h.data(), h.size(), s);
}

}  // namespace

bool device_enumeration(gale_ctx *ctx, uint64_t gen, const int32_t **E, const int32_t **F) {
    if (!ctx->cb || ctx->cb->dev_gen != gen || !ctx->cb->E || !ctx->cb->F) return false;
    *E = ctx->cb->E;
    *F = ctx->cb->F;
    return true;
}

// Sorted enumeration on the device (declared in gale_enum.h).
gale_status enumerate_sorted_device(gale_ctx *ctx, uint64_t gen, std::vector<int64_t> &IE,
                                    std::vector<int64_t> &IF) {
    if (ctx->device < 0 || (ctx->precond & GALE_ET) == 0) return GALE_ENOTFOUND;
    gale_status st = gale_build_clusters(ctx, nullptr, 0, GALE_ET, GALE_MODE_BATCHED);
    if (st == GALE_OK) st = gale_synchronize(ctx);
    if (st != GALE_OK) return st;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(GALE_ECUDA, "cudaSetDevice");
    cudaStream_t s = ctx->stream;
    const HostMesh &hm = ctx->hm;
    const int32_t K = hm.K;
    IE.assign(size_t(K) + 1, 0);
    for (int32_t k = 0; k < K; ++k) IE[k + 1] = IE[k] + ctx->sizes[size_t(5) * k + 2];
    const int64_t nE = IE[K];
    if (nE >= INT32_MAX) return fail(GALE_EINVAL, "more than 2^31 - 1 edges");
    if (!ctx->cb) ctx->cb = new Cobound();
    Cobound &cb = *ctx->cb;
    if (!cb.rows) {
        cb.rows = upload(ctx, hm.rows, s);
        cb.cluster_of = upload(ctx, hm.cluster_of, s);
        if (!cb.rows || !cb.cluster_of) return fail(GALE_ENOMEM, "device allocation of the mesh rows failed");
    }
    std::vector<int64_t> base(ctx->bulk_offs.begin(), ctx->bulk_offs.begin() + size_t(10) * K);
    std::vector<void *> tmp;
    auto dal = [&](size_t bytes) {
        void *p = ctx->dalloc(std::max<size_t>(bytes, 16));
        if (p) tmp.push_back(p);
        return p;
    };
    auto release = [&]() {
        for (void *p : tmp) ctx->dfree(p);
        tmp.clear();
    };
    int64_t *d_base = static_cast<int64_t *>(dal(base.size() * 8));
    int64_t *d_IE = static_cast<int64_t *>(dal(IE.size() * 8));
    int32_t *d_E = static_cast<int32_t *>(dal(size_t(2) * nE * 4));
    int32_t *d_nf = static_cast<int32_t *>(dal(size_t(nE) * 4 + 4));
    int32_t *d_FS = static_cast<int32_t *>(dal((size_t(nE) + 1) * 4));
    int64_t *d_IF = static_cast<int64_t *>(dal((size_t(K) + 1) * 8));
    const int64_t nb = (nE + kThreads - 1) / kThreads;
    int64_t *d_bsum = static_cast<int64_t *>(dal((size_t(nb) + 1) * 8));
    if (!d_base || !d_IE || !d_E || !d_nf || !d_FS || !d_IF || !d_bsum) {
        release();
        return fail(GALE_ENOMEM, "device allocation for the enumeration failed");
    }
    cudaMemcpyAsync(d_base, base.data(), base.size() * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_IE, IE.data(), IE.size() * 8, cudaMemcpyHostToDevice, s);
    CbMesh m{};
    m.rows = reinterpret_cast<const int4 *>(cb.rows);
    m.cluster_of = cb.cluster_of;
    m.I_V = ctx->d_I_V;
    m.IE = d_IE;
    m.et_uoff = ctx->bulk[B_ET_UOFF];
    m.et_w = ctx->bulk[B_ET_W];
    m.et_off = ctx->bulk[B_ET_OFF];
    m.et_val = ctx->bulk[B_ET_VAL];
    m.base = d_base;
    m.sizes = ctx->d_sizes;
    m.nv = hm.nv;
    m.nE = nE;
    const int sms = ctx->sm_count > 0 ? ctx->sm_count : 1;
    auto grid_for = [&](int64_t n) {
        return int(std::min<int64_t>(std::max<int64_t>((n + kThreads - 1) / kThreads, 1), int64_t(sms) * 16));
    };
    k_enum_edges<<<grid_for(hm.nv), kThreads, 0, s>>>(m, d_E);
    k_enum_faces<false><<<grid_for(nE), kThreads, 0, s>>>(m, d_E, d_nf, nullptr, nullptr, ctx->d_err);
    if (nb > 0) {
        scan_sums<<<int(nb), kThreads, 0, s>>>(d_nf, nE, d_bsum);
        scan_bsums<<<1, kThreads, 0, s>>>(d_bsum, nb);
        scan_write<<<int(nb), kThreads, 0, s>>>(d_nf, nE, d_bsum, d_FS, nb, ctx->d_err);
    } else {
        cudaMemsetAsync(d_FS, 0, 4, s);
    }
    int32_t nF = 0;
    if (cudaMemcpyAsync(&nF, d_FS + nE, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        release();
        return fail(GALE_ECUDA, "enumeration count pass failed");
    }
    int32_t e = 0;
    cudaMemcpy(&e, ctx->d_err, 4, cudaMemcpyDeviceToHost);
    if (e) {
        cudaMemset(ctx->d_err, 0, 4);
        release();
        return fail(GALE_EDEVICE, "enumeration count pass: error word " + std::to_string(e));
    }
    int32_t *d_F = static_cast<int32_t *>(dal(size_t(3) * nF * 4));
    if (!d_F) {
        release();
        return fail(GALE_ENOMEM, "device allocation of the triangle list failed");
    }
    k_enum_faces<true><<<grid_for(nE), kThreads, 0, s>>>(m, d_E, nullptr, d_FS, d_F, ctx->d_err);
    k_enum_if<<<grid_for(K + 1), kThreads, 0, s>>>(d_IE, d_FS, K, d_IF);
    // only the intervals come to the host; E and F are copied by the
    // queries that need them (gale_get_enumeration, gale_boundary)
    IF.assign(size_t(K) + 1, 0);
    const gale_status cst = copy_to_host(ctx, IF.data(), d_IF, IF.size() * 8);
    if (cst != GALE_OK) {
        release();
        return cst;
    }
    cudaMemcpy(&e, ctx->d_err, 4, cudaMemcpyDeviceToHost);
    if (e) {
        cudaMemset(ctx->d_err, 0, 4);
        release();
        return fail(GALE_EDEVICE, "enumeration fill pass: error word " + std::to_string(e));
    }
    // the device lists stay with the coboundary pass, which would otherwise
    // upload the same arrays again
    for (int32_t **p : {&cb.E, &cb.F, &cb.ebk, &cb.fbk})
        if (*p) {
            ctx->dfree(*p);
            *p = nullptr;
        }
    for (int64_t **p : {&cb.IE, &cb.IF})
        if (*p) {
            ctx->dfree(*p);
            *p = nullptr;
        }
    cb.E = d_E;
    cb.F = d_F;
    cb.IE = d_IE;
    cb.IF = d_IF;
    cb.dev_gen = gen;
    tmp.erase(std::remove_if(tmp.begin(), tmp.end(),
                             [&](void *p) { return p == d_E || p == d_F || p == d_IE || p == d_IF; }),
              tmp.end());
    release();
    return GALE_OK;
}

}  // namespace gale

extern "C" gale_status gale_build_coboundary(gale_ctx *ctx, uint32_t which, gale_coboundary *out) {
    using namespace gale;
    if (!ctx || !out) return fail(GALE_EINVAL, "NULL argument");
    if (ctx->device < 0) return fail(GALE_EINVAL, "host-only context");
    if (which == 0 || (which & ~uint32_t(GALE_CB_VE | GALE_CB_VF | GALE_CB_EF | GALE_CB_FT)))
        return fail(GALE_EINVAL, "which must be a non-empty set of GALE_CB_* bits");
    const uint32_t need = GALE_VT | GALE_VV | GALE_ET;
    if ((ctx->precond & need) != need)
        return fail(GALE_EINVAL, "coboundary relations need VT, VV and ET in the precondition mask");
    EnumView ev{};
    if (!enumeration_view(ctx, &ev)) return fail(GALE_ENOTFOUND, "no enumeration: call gale_enumerate first");
    const int64_t nE = ev.nE, nF = ev.nF;
    const uint64_t gen = ev.gen;
    if (nE >= INT32_MAX || nF >= INT32_MAX) return fail(GALE_EINVAL, "more than 2^31 - 1 edges or triangles");
    // the stars, neighbour sets and edge stars of every vertex
    gale_status st = gale_build_clusters(ctx, nullptr, 0, need, GALE_MODE_BATCHED);
    if (st != GALE_OK) return st;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(GALE_ECUDA, "cudaSetDevice");
    cudaStream_t s = ctx->stream;
    const HostMesh &hm = ctx->hm;
    const int32_t K = hm.K;
    if (!ctx->cb) ctx->cb = new Cobound();
    Cobound &cb = *ctx->cb;
    if (!cb.rows) {
        cb.rows = upload(ctx, hm.rows, s);
        cb.cluster_of = upload(ctx, hm.cluster_of, s);
        if (!cb.rows || !cb.cluster_of) return fail(GALE_ENOMEM, "device allocation of the mesh rows failed");
    }
    // bases of every cluster's segments in the bulk arrays
    std::vector<int64_t> base(ctx->bulk_offs.begin(), ctx->bulk_offs.begin() + size_t(10) * K);
    if (cb.base) ctx->dfree(cb.base);
    cb.base = upload(ctx, base, s);
    if (!cb.base) return fail(GALE_ENOMEM, "device allocation failed");
    CbMesh m{reinterpret_cast<const int4 *>(cb.rows), cb.cluster_of, ctx->d_I_V, cb.E, cb.F, cb.ebk, cb.fbk,
             cb.IE, cb.IF, cb.eo, cb.ekw, cb.feo, cb.fkc, cb.e2s, cb.f2s,
             ctx->bulk[B_VT_OFF], ctx->bulk[B_VT_VAL], ctx->bulk[B_VV_OFF], ctx->bulk[B_VV_VAL],
             ctx->bulk[B_ET_W], ctx->bulk[B_ET_OFF], ctx->bulk[B_ET_VAL], ctx->bulk[B_ET_UOFF], nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, cb.base, ctx->d_sizes,
             hm.nv, nE, nF, cb.sorted_ids};
    const int sms = ctx->sm_count > 0 ? ctx->sm_count : 1;
    auto grid_for = [&](int64_t n) {
        return int(std::min<int64_t>(std::max<int64_t>((n + kThreads - 1) / kThreads, 1), int64_t(sms) * 16));
    };
    if (cb.enm_gen != gen) {
        for (int32_t **p : {&cb.eo, &cb.ekw, &cb.feo, &cb.fkc, &cb.fo, &cb.e2s, &cb.f2s})
            if (*p) {
                ctx->dfree(*p);
                *p = nullptr;
            }
        cb.enm_gen = 0;
        if (cb.dev_gen != gen) {  // the lists are not on the device yet
            if (!ev.E || !ev.F) return fail(GALE_EINVAL, "the enumeration's lists are gone from the device");
            for (int32_t **p : {&cb.E, &cb.F, &cb.ebk, &cb.fbk})
                if (*p) {
                    ctx->dfree(*p);
                    *p = nullptr;
                }
            for (int64_t **p : {&cb.IE, &cb.IF})
                if (*p) {
                    ctx->dfree(*p);
                    *p = nullptr;
                }
            cb.dev_gen = 0;
            cb.E = upload(ctx, ev.E, size_t(2) * nE, s);
            cb.F = upload(ctx, ev.F, size_t(3) * nF, s);
            if (ev.ebk) cb.ebk = upload(ctx, ev.ebk, size_t(nE), s);
            if (ev.fbk) cb.fbk = upload(ctx, ev.fbk, size_t(nF), s);
            cb.IE = upload(ctx, ev.IE, size_t(K) + 1, s);
            cb.IF = upload(ctx, ev.IF, size_t(K) + 1, s);
            if (!cb.E || !cb.F || (ev.ebk && !cb.ebk) || (ev.fbk && !cb.fbk) || !cb.IE || !cb.IF)
                return fail(GALE_ENOMEM, "device allocation of the enumeration failed");
            cb.dev_gen = gen;
        }
        auto dal = [&](int64_t n) { return static_cast<int32_t *>(ctx->dalloc(size_t(std::max<int64_t>(n, 1)) * 4)); };
        cb.eo = dal(hm.nv + 1);
        cb.fo = dal(hm.nv + 1);
        cb.ekw = dal(nE);
        cb.e2s = dal(nE);
        cb.feo = dal(nE + 1);
        cb.fkc = dal(nF);
        cb.f2s = dal(nF);
        if (!cb.eo || !cb.fo || !cb.ekw || !cb.e2s || !cb.feo || !cb.fkc || !cb.f2s)
            return fail(GALE_ENOMEM, "device allocation of the enumeration index failed");
        // ids follow the vertex-tuple order exactly when no key arrays exist
        cb.sorted_ids = ev.ebk == nullptr;
        m.E = cb.E;
        m.F = cb.F;
        m.ebk = cb.ebk;
        m.fbk = cb.fbk;
        m.IE = cb.IE;
        m.IF = cb.IF;
        m.sorted_ids = cb.sorted_ids;
        k_eo<<<grid_for(hm.nv + 1), kThreads, 0, s>>>(m, cb.eo);
        k_fo<<<grid_for(hm.nv + 1), kThreads, 0, s>>>(m, cb.fo);
        k_keys<<<grid_for(std::max(nE, nF)), kThreads, 0, s>>>(m, cb.ekw, cb.e2s, cb.fkc, cb.f2s);
        k_feo<<<grid_for(nE + 1), kThreads, 0, s>>>(m, cb.fo, cb.feo);
        if (cudaGetLastError() != cudaSuccess) return fail(GALE_ECUDA, "coboundary lookup-structure launch failed");
        cb.enm_gen = gen;
    }
    m.eo = cb.eo;
    m.ekw = cb.ekw;
    m.feo = cb.feo;
    m.fkc = cb.fkc;
    m.e2s = cb.e2s;
    m.f2s = cb.f2s;
    m.sorted_ids = cb.sorted_ids;
    const int64_t rows_of[4] = {hm.nv, hm.nv, nE, nF};
    // VF is read from VE (in VV order) and EF: those two first, and built
    // whenever VF is asked for
    const uint32_t build = which | ((which & GALE_CB_VF) ? uint32_t(GALE_CB_VE | GALE_CB_EF) : 0u);
    m.ef_off = nullptr;
    m.ef_val = nullptr;
    m.ve_off = nullptr;
    m.ve_val = nullptr;
    m.ef_third = nullptr;
    m.third_out = nullptr;
    for (int rel : {int(REL_VE), int(REL_EF), int(REL_VF), int(REL_FT)}) {
        if (!(build & (1u << rel))) continue;
        const int64_t n = rows_of[rel];
        const int64_t nb = (n + kThreads - 1) / kThreads;
        if (!grow(ctx, cb.cnt, cb.cnt_cap, std::max<int64_t>(n, 1)) ||
            !grow(ctx, cb.bsum, cb.bsum_cap, nb + 1) || !grow(ctx, cb.off[rel], cb.off_cap[rel], n + 1))
            return fail(GALE_ENOMEM, "device allocation of coboundary counts failed");
        const int grid = grid_for(n);
        switch (rel) {
            case REL_VE: cb_count<REL_VE><<<grid, kThreads, 0, s>>>(m, n, cb.cnt, ctx->d_err); break;
            case REL_VF: cb_count<REL_VF><<<grid, kThreads, 0, s>>>(m, n, cb.cnt, ctx->d_err); break;
            case REL_EF: cb_count<REL_EF><<<grid, kThreads, 0, s>>>(m, n, cb.cnt, ctx->d_err); break;
            default: cb_count<REL_FT><<<grid, kThreads, 0, s>>>(m, n, cb.cnt, ctx->d_err); break;
        }
        if (nb > 0) {
            scan_sums<<<int(nb), kThreads, 0, s>>>(cb.cnt, n, cb.bsum);
            scan_bsums<<<1, kThreads, 0, s>>>(cb.bsum, nb);
            scan_write<<<int(nb), kThreads, 0, s>>>(cb.cnt, n, cb.bsum, cb.off[rel], nb, ctx->d_err);
        } else {
            cudaMemsetAsync(cb.off[rel], 0, sizeof(int32_t), s);
        }
        int32_t total = 0;
        if (cudaMemcpyAsync(&total, cb.off[rel] + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(GALE_ECUDA, "coboundary count pass failed");
        int32_t e = 0;
        cudaMemcpy(&e, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e) {
            cudaMemset(ctx->d_err, 0, sizeof(int32_t));
            return fail(GALE_EDEVICE, "coboundary count pass: error word " + std::to_string(e));
        }
        if (!grow(ctx, cb.val[rel], cb.val_cap[rel], std::max<int64_t>(total, 1)) ||
            (rel == REL_EF && !grow(ctx, cb.ef_third, cb.ef_third_cap, std::max<int64_t>(total, 1))))
            return fail(GALE_ENOMEM, "device allocation of coboundary values failed");
        m.third_out = cb.ef_third;
        switch (rel) {
            case REL_VE: cb_fill<REL_VE><<<grid, kThreads, 0, s>>>(m, n, cb.off[rel], cb.val[rel], ctx->d_err); break;
            case REL_VF: cb_fill<REL_VF><<<grid, kThreads, 0, s>>>(m, n, cb.off[rel], cb.val[rel], ctx->d_err); break;
            case REL_EF: cb_fill<REL_EF><<<grid, kThreads, 0, s>>>(m, n, cb.off[rel], cb.val[rel], ctx->d_err); break;
            default: cb_fill<REL_FT><<<grid, kThreads, 0, s>>>(m, n, cb.off[rel], cb.val[rel], ctx->d_err); break;
        }
        if (cudaGetLastError() != cudaSuccess) return fail(GALE_ECUDA, "coboundary launch failed");
        cb.rows_of[rel] = n;
        cb.len[rel] = total;
        if (rel == REL_EF) {
            m.ef_off = cb.off[REL_EF];
            m.ef_val = cb.val[REL_EF];
            m.ef_third = cb.ef_third;
        }
        if (rel == REL_VE) {
            m.ve_off = cb.off[REL_VE];
            m.ve_val = cb.val[REL_VE];
        }
    }
    // VE rows are ascending already with the sorted numbering
    if ((build & GALE_CB_VE) && !cb.sorted_ids && hm.nv > 0)
        cb_sort_rows<<<grid_for(hm.nv), kThreads, 0, s>>>(hm.nv, cb.off[REL_VE], cb.val[REL_VE]);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(GALE_ECUDA, "cudaStreamSynchronize");
    int32_t e = 0;
    cudaMemcpy(&e, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e) {
        cudaMemset(ctx->d_err, 0, sizeof(int32_t));
        return fail(GALE_EDEVICE, "coboundary fill pass: error word " + std::to_string(e));
    }
    for (int rel = 0; rel < 4; ++rel) {
        const bool have = (which & (1u << rel)) != 0;
        out->rows[rel] = have ? cb.rows_of[rel] : 0;
        out->len[rel] = have ? cb.len[rel] : 0;
        out->off[rel] = have ? cb.off[rel] : nullptr;
        out->val[rel] = have ? cb.val[rel] : nullptr;
    }
    return GALE_OK;
}
