// Coboundary relations VE, VF, EF, FT in the ids of the edge / triangle
// enumeration (Section 4.4: coboundary relations are computed by the GPU for
// whole segments; Section 5 evaluates VE, VF, EF and FT among them).
//
// Inputs on the device: the canonical tet rows, each vertex's cluster and
// the enumeration (E, F, I_E, I_F and each segment's ids in vertex-tuple
// order).  The enumeration itself, when made on the device, reads every
// cluster's ET rows from a batched build (enumerate_sorted_device).
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
// (a, b, c) among the few triangles over its edge (a, b).
//
// The relations are scattered from the simplices (details at the scatter
// kernels below): every row is a contiguous range of the sorted order (VE(v):
// v's upper edges; EF(e): the triangles over e; VF(v): the triangles with
// lowest vertex v) plus entries that other edges and triangles place by
// atomic cursors after counts and an exclusive scan; FT takes two slots per
// triangle that its tets claim (a counted form with cursors and row sorts
// when a triangle lies in three or more tets).  With the sorted numbering
// only each row's scattered prefix needs sorting, and VF is gathered from VE
// and EF; otherwise rows are sorted whole.
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

    int32_t *cnt = nullptr;        // counts of the largest relation
    int64_t *bsum = nullptr;       // scan block sums
    int64_t cnt_cap = 0, bsum_cap = 0;
    int32_t *off[4] = {}, *val[4] = {};
    int32_t *scratch = nullptr;    // counters and lookups of the scatter passes
    int64_t scratch_cap = 0;
    int64_t off_cap[4] = {}, val_cap[4] = {};
    int64_t rows_of[4] = {}, len[4] = {};
    bool ft_general = false;       // FT by counts and cursors: some triangle lies in three or more tets
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
    // the ET rows of a batched build (the sorted enumeration reads them)
    const int32_t *et_w, *et_off, *et_val;
    const int32_t *et_uoff;          // ET edges per own lower vertex
    const int64_t *base;
    const int64_t *sizes;  // [K][5] per-cluster entries: VT, VV, edges, ET, TT
    int64_t nv, nE, nF;
    bool sorted_ids;
};

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

// ---- the relations by scatter, over sorted positions ----
// Every row is [scattered part | contiguous part].  The contiguous part is a
// range the vertex-tuple order gives whole: for VE(v) the edges whose lower
// vertex is v (sorted positions eo[v] ..), for EF(e) the triangles whose
// first two vertices are e (feo[e] ..), for VF(v) the triangles whose lowest
// vertex is v (fo[v] ..).  The other entries come from the edges, triangles
// and tets that hold the row's simplex elsewhere than in front: an edge
// (a, b) is in VE(b); a triangle (a, b, c) is in EF(a, c), EF(b, c), VF(b)
// and VF(c); a tet is in FT of its four faces.  They take slots by atomic
// counters, and a last pass sorts every row by id.  With the sorted
// numbering the scattered ids all precede the contiguous ones, so only the
// scattered prefix moves.

__device__ __forceinline__ int64_t erow(const CbMesh &m, int64_t j) { return m.sorted_ids ? j : m.ebk[j]; }
__device__ __forceinline__ int64_t frow(const CbMesh &m, int64_t p) { return m.sorted_ids ? p : m.fbk[p]; }

struct Scatter {
    int32_t *ve_n, *ve_fill;               // [nv] lower edges of v, and the cursor of their slots
    int32_t *ef_lo, *ef_mid;               // [nE] (sorted positions) triangles (x, u, w), x < u, and
                                           // (u, x, w), u < x < w, of edge (u, w)
    int32_t *ef_lofill, *ef_midfill;       // [nE] cursors of their slots
    int32_t *vf_n, *vf_fill;               // [nv] triangles with v as second or third vertex; cursor
    int32_t *tri_ac, *tri_bc;              // [nF] sorted positions of the edges (a, c), (b, c) of triangle p
    int2 *ft_slot;                         // [nF] (sorted positions) the one or two tets of a triangle
    int2 *ef_tail;                         // [nE] (sorted numbering, VF gather) EF(j) after its lower part
    int32_t *cnt;                          // row lengths of the relation being placed
    const int32_t *ve_off, *ef_off, *vf_off, *ft_off;
    int32_t *ve_val, *ef_val, *vf_val, *ft_val;
};

// edges: VE(b) of every edge (a, b); FILL also writes the contiguous parts
template <bool FILL>
__global__ void __launch_bounds__(kThreads) k_sc_edges(CbMesh m, Scatter sc, int32_t *err) {
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < m.nE; j += int64_t(gridDim.x) * blockDim.x) {
        const int32_t id = edge_id(m, j);
        const int32_t a = m.E[2 * int64_t(id)], b = m.E[2 * int64_t(id) + 1];
        if (!FILL) {
            atomicAdd(&sc.ve_n[b], 1);
            continue;
        }
        sc.ve_val[sc.ve_off[a] + sc.ve_n[a] + (j - m.eo[a])] = id;
        sc.ve_val[atomicAdd(&sc.ve_fill[b], 1)] = id;
    }
}

// triangles: EF(a, c), EF(b, c), VF(b), VF(c) of every triangle (a, b, c)
template <bool FILL>
__global__ void __launch_bounds__(kThreads) k_sc_tris(CbMesh m, Scatter sc, bool ef, bool vf, int32_t *err) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < m.nF; p += int64_t(gridDim.x) * blockDim.x) {
        const int32_t id = face_id(m, p);
        const int32_t *t = m.F + 3 * int64_t(id);
        const int32_t b = t[1], c = t[2];
        if (!FILL) {
            if (ef) {
                const int32_t a = t[0];
                const int64_t jac = epos(m, a, c), jbc = epos(m, b, c);
                if (jac < 0 || jbc < 0) {
                    atomicOr(err, ERR_BAD_BLOCK);
                    sc.tri_ac[p] = sc.tri_bc[p] = -1;
                } else {
                    sc.tri_ac[p] = int32_t(jac);
                    sc.tri_bc[p] = int32_t(jbc);
                    atomicAdd(&sc.ef_mid[jac], 1);
                    atomicAdd(&sc.ef_lo[jbc], 1);
                }
            }
            if (vf) {
                atomicAdd(&sc.vf_n[b], 1);
                atomicAdd(&sc.vf_n[c], 1);
            }
            continue;
        }
        if (ef) {
            const int32_t jac = sc.tri_ac[p], jbc = sc.tri_bc[p];
            if (jac >= 0 && jbc >= 0) {
                sc.ef_val[atomicAdd(&sc.ef_midfill[jac], 1)] = id;
                sc.ef_val[atomicAdd(&sc.ef_lofill[jbc], 1)] = id;
            }
        }
        if (vf) {
            sc.vf_val[atomicAdd(&sc.vf_fill[b], 1)] = id;
            sc.vf_val[atomicAdd(&sc.vf_fill[c], 1)] = id;
        }
    }
}
// FT: a triangle lies in one or two tets, so each has two slots (sorted
// position order); every tet claims a slot of each of its four faces, and
// a pass over the triangles writes the rows (smaller tet first)
__device__ __forceinline__ void ft_claim(int2 *slot, int32_t q, int32_t t, int32_t *err) {
    if (atomicCAS(&slot[q].x, -1, t) == -1) return;
    if (atomicCAS(&slot[q].y, -1, t) != -1) atomicOr(err, ERR_NONMANIFOLD);
}
// MODE: FT_SLOTS claims the two slots; FT_COUNT counts each triangle's tets
// (sc.cnt, by row); FT_FILL places them by cursors (sc.cnt zeroed) in rows
// that a sort then orders - the form for a mesh with a triangle in three
// or more tets.
enum { FT_SLOTS = 0, FT_COUNT = 1, FT_FILL = 2 };
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_ft_tets(CbMesh m, Scatter sc, int64_t nT, int32_t *err) {
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nT; t += int64_t(gridDim.x) * blockDim.x) {
        const int4 r = m.rows[t];
        const int64_t jab = epos(m, r.x, r.y), jac = epos(m, r.x, r.z), jbc = epos(m, r.y, r.z);
        const int64_t f0 = jab < 0 ? -1 : fpos_at(m, jab, r.z), f1 = jab < 0 ? -1 : fpos_at(m, jab, r.w);
        const int64_t f2 = jac < 0 ? -1 : fpos_at(m, jac, r.w), f3 = jbc < 0 ? -1 : fpos_at(m, jbc, r.w);
        if (f0 < 0 || f1 < 0 || f2 < 0 || f3 < 0) {
            atomicOr(err, ERR_BAD_BLOCK);
            continue;
        }
        const int64_t f[4] = {f0, f1, f2, f3};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (MODE == FT_SLOTS) {
                ft_claim(sc.ft_slot, int32_t(f[q]), int32_t(t), err);
            } else {
                const int64_t row = frow(m, f[q]);
                const int32_t c = atomicAdd(&sc.cnt[row], 1);
                if (MODE == FT_FILL) sc.ft_val[sc.ft_off[row] + c] = int32_t(t);
            }
        }
    }
}
__global__ void __launch_bounds__(kThreads) k_len_ft(CbMesh m, Scatter sc, int32_t *err) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < m.nF; p += int64_t(gridDim.x) * blockDim.x) {
        const int2 q = sc.ft_slot[p];
        if (q.x < 0) atomicOr(err, ERR_BAD_BLOCK);  // a triangle in no tet
        sc.cnt[frow(m, p)] = (q.x >= 0) + (q.y >= 0);
    }
}
__global__ void __launch_bounds__(kThreads) k_ft_write(CbMesh m, Scatter sc) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < m.nF; p += int64_t(gridDim.x) * blockDim.x) {
        const int2 q = sc.ft_slot[p];
        int32_t *o = sc.ft_val + sc.ft_off[frow(m, p)];
        if (q.y < 0) {
            if (q.x >= 0) o[0] = q.x;
        } else {
            o[0] = min(q.x, q.y);
            o[1] = max(q.x, q.y);
        }
    }
}

// row lengths: scattered part + contiguous part
__global__ void __launch_bounds__(kThreads) k_len_ve(CbMesh m, Scatter sc) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < m.nv; v += int64_t(gridDim.x) * blockDim.x)
        sc.cnt[v] = sc.ve_n[v] + (m.eo[v + 1] - m.eo[v]);
}
__global__ void __launch_bounds__(kThreads) k_len_vf(CbMesh m, Scatter sc, const int32_t *fo) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < m.nv; v += int64_t(gridDim.x) * blockDim.x)
        sc.cnt[v] = sc.vf_n[v] + (fo[v + 1] - fo[v]);
}
__global__ void __launch_bounds__(kThreads) k_len_ef(CbMesh m, Scatter sc) {
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < m.nE; j += int64_t(gridDim.x) * blockDim.x)
        sc.cnt[erow(m, j)] = sc.ef_lo[j] + sc.ef_mid[j] + (m.feo[j + 1] - m.feo[j]);
}

// Row sorts.  Only a row's first plen entries need ordering: with the
// sorted numbering the scattered entries all precede (and are smaller than)
// the contiguous part, so plen is the scattered count; otherwise it is the
// whole row.
enum { PL_VE = 0, PL_VF = 1, PL_EF = 2, PL_FULL = 3 };
__device__ __forceinline__ void insertion_sort(int32_t *o, int32_t n) {
    for (int32_t i = 1; i < n; ++i) {
        const int32_t y = o[i];
        int32_t j = i - 1;
        while (j >= 0 && o[j] > y) {
            o[j + 1] = o[j];
            --j;
        }
        o[j + 1] = y;
    }
}

// ascending bitonic sort of N values held in registers (all indices are
// compile-time constants once unrolled)
template <int N>
__device__ __forceinline__ void bitonic_regs(int32_t (&x)[N]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const int32_t a = x[i], b = x[l];
                    const bool asc = (i & k) == 0;
                    x[i] = asc ? min(a, b) : max(a, b);
                    x[l] = asc ? max(a, b) : min(a, b);
                }
            }
}

// one thread per row: prefixes of up to N entries are sorted in registers,
// longer ones in place.  A block's rows are one contiguous span of the
// values: it is staged through shared memory when it fits, so that loads
// and stores are coalesced.  FRONT writes the row's contiguous part first
// (EF: the triangles over the edge; VF: the triangles with lowest vertex v).
enum { FRONT_NONE = 0, FRONT_EF = 1, FRONT_VF = 2 };
// SPAN: int32 entries of a staged span (0: rows are sorted where they are).
// With the sorted numbering, EF's sort also records for each edge the range
// of its entries after the lower part (the VF gather reads them).
template <int PL, int N, int FRONT, int SPAN>
__global__ void __launch_bounds__(kThreads) k_sort_rows(CbMesh m, Scatter sc, int64_t rows, const int32_t *off,
                                                        int32_t *val, const int32_t *fo) {
    __shared__ int32_t s_val[SPAN > 0 ? SPAN : 1];
    for (int64_t r0 = int64_t(blockIdx.x) * kThreads; r0 < rows; r0 += int64_t(gridDim.x) * kThreads) {
        const int64_t r1 = min(rows, r0 + kThreads);
        const int32_t base = off[r0], span = off[r1] - base;
        const bool staged = SPAN > 0 && span <= SPAN;
        if (staged) {
            for (int32_t u = threadIdx.x; u < span; u += kThreads) s_val[u] = val[base + u];
            __syncthreads();
        }
        const int64_t r = r0 + threadIdx.x;
        if (r < r1) {
            int32_t *o = staged ? s_val + (off[r] - base) : val + off[r];
            const int32_t len = off[r + 1] - off[r];
            if (FRONT == FRONT_EF) {
                const int64_t j = m.sorted_ids ? r : m.e2s[r];
                if (m.sorted_ids && sc.ef_tail) sc.ef_tail[j] = make_int2(off[r] + sc.ef_lo[j], off[r + 1]);
                int32_t *f = o + sc.ef_lo[j] + sc.ef_mid[j];
                const int32_t p0 = m.feo[j], p1 = m.feo[j + 1];
                for (int32_t p = p0; p < p1; ++p) f[p - p0] = face_id(m, p);
            } else if (FRONT == FRONT_VF) {
                int32_t *f = o + sc.vf_n[r];
                const int32_t p0 = fo[r], p1 = fo[r + 1];
                for (int32_t p = p0; p < p1; ++p) f[p - p0] = face_id(m, p);
            }
            int32_t n;
            if (!m.sorted_ids || PL == PL_FULL) n = len;
            else if (PL == PL_VE) n = sc.ve_n[r];
            else if (PL == PL_VF) n = sc.vf_n[r];
            else n = sc.ef_lo[r] + sc.ef_mid[r];
            if (n > N) {
                insertion_sort(o, n);
            } else if (n >= 2) {
                int32_t x[N];
#pragma unroll
                for (int i = 0; i < N; ++i) x[i] = i < n ? o[i] : INT32_MAX;
                bitonic_regs<N>(x);
#pragma unroll
                for (int i = 0; i < N; ++i)
                    if (i < n) o[i] = x[i];
            }
        }
        if (staged) {
            __syncthreads();
            for (int32_t u = threadIdx.x; u < span; u += kThreads) val[base + u] = s_val[u];
            __syncthreads();
        }
    }
}

// VF with the sorted numbering, from VE and EF (both sorted): the triangles
// through v whose lowest vertex a is not v are, for the lower edges (a, v)
// in ascending a, EF(a, v) after its lower part - its middle part (a, x, v)
// and its contiguous part (a, v, x) - already in id order; the triangles
// with lowest vertex v follow.
// counts: edge (a, b) gives VF(b) its middle and contiguous EF entries
__global__ void __launch_bounds__(kThreads) k_vf_count_sorted(CbMesh m, Scatter sc) {
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < m.nE; j += int64_t(gridDim.x) * blockDim.x) {
        const int32_t b = m.E[2 * j + 1];  // sorted numbering: edge id j is sorted position j
        atomicAdd(&sc.vf_n[b], sc.ef_mid[j] + (m.feo[j + 1] - m.feo[j]));
    }
}
constexpr int kGatherSpan = 12288;
__global__ void __launch_bounds__(kThreads) k_vf_gather(CbMesh m, Scatter sc, const int32_t *fo) {
    __shared__ int32_t s_val[kGatherSpan];  // the block's rows, stored coalesced
    for (int64_t v0 = int64_t(blockIdx.x) * kThreads; v0 < m.nv; v0 += int64_t(gridDim.x) * kThreads) {
        const int64_t v1 = min(m.nv, v0 + kThreads);
        const int32_t base = sc.vf_off[v0], span = sc.vf_off[v1] - base;
        const bool staged = span <= kGatherSpan;
        const int64_t v = v0 + threadIdx.x;
        if (v < v1) {
            const int32_t *ve = sc.ve_val + sc.ve_off[v];
            const int32_t nl = sc.ve_n[v];
            int32_t *o = staged ? s_val + (sc.vf_off[v] - base) : sc.vf_val + sc.vf_off[v];
            for (int32_t q = 0; q < nl; ++q) {
                const int2 t = sc.ef_tail[ve[q]];
                for (int32_t i = t.x; i < t.y; ++i) *o++ = sc.ef_val[i];
            }
            const int32_t p0 = fo[v], p1 = fo[v + 1];
            for (int32_t p = p0; p < p1; ++p) *o++ = p;
        }
        if (staged) {
            __syncthreads();
            for (int32_t u = threadIdx.x; u < span; u += kThreads) sc.vf_val[base + u] = s_val[u];
            __syncthreads();
        }
    }
}

// fill cursors: every scattered part's first slot, so that a scatter is
// one atomic and one store
__global__ void __launch_bounds__(kThreads) k_cursors(CbMesh m, Scatter sc, bool ve, bool vf, bool ef) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t v = t0; v < m.nv; v += stride) {
        if (ve) sc.ve_fill[v] = sc.ve_off[v];
        if (vf) sc.vf_fill[v] = sc.vf_off[v];
    }
    if (ef)
        for (int64_t j = t0; j < m.nE; j += stride) {
            const int32_t o = sc.ef_off[erow(m, j)];
            sc.ef_lofill[j] = o;
            sc.ef_midfill[j] = o + sc.ef_lo[j];
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

// exclusive scan of cnt[0..n) into off[0..n], in tiles of kScanTile counts
// (kScanItems consecutive ones per thread): tile sums, one pass over the
// tile sums, then the per-tile scans
constexpr int kScanItems = 16;
constexpr int64_t kScanTile = int64_t(kThreads) * kScanItems;
inline int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// the sum of a thread's kScanItems counts, from i0
__device__ __forceinline__ int64_t items_sum(const int32_t *cnt, int64_t n, int64_t i0) {
    int64_t t = 0;
    if (i0 + kScanItems <= n && (i0 & 3) == 0) {
        const int4 *q = reinterpret_cast<const int4 *>(cnt + i0);
#pragma unroll
        for (int u = 0; u < kScanItems / 4; ++u) {
            const int4 v = q[u];
            t += int64_t(v.x) + v.y + v.z + v.w;
        }
    } else {
        for (int64_t i = i0; i < min(n, i0 + kScanItems); ++i) t += cnt[i];
    }
    return t;
}

// block-wide inclusive scan of one int64 per thread
__device__ __forceinline__ int64_t block_incl_scan(int64_t x, int64_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kThreads / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    return x + (warp > 0 ? s_warp[warp - 1] : 0);
}

__global__ void __launch_bounds__(kThreads) scan_sums(const int32_t *cnt, int64_t n, int64_t *bsum) {
    __shared__ int64_t s_warp[kThreads / 32];
    const int64_t i0 = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    const int64_t tot = block_incl_scan(items_sum(cnt, n, i0), s_warp);
    if (threadIdx.x == kThreads - 1) bsum[blockIdx.x] = tot;
}

// exclusive scan of the nb tile sums in place (bsum[nb] = total), one
// block: each thread sums a contiguous chunk, the chunk totals are scanned,
// then each thread rewrites its chunk
__global__ void __launch_bounds__(kThreads) scan_bsums(int64_t *bsum, int64_t nb) {
    __shared__ int64_t s_warp[kThreads / 32];
    const int64_t per = (nb + kThreads - 1) / kThreads;
    const int64_t b0 = min(nb, int64_t(threadIdx.x) * per), b1 = min(nb, b0 + per);
    int64_t sum = 0;
    for (int64_t b = b0; b < b1; ++b) sum += bsum[b];
    const int64_t incl = block_incl_scan(sum, s_warp);
    int64_t run = incl - sum;
    for (int64_t b = b0; b < b1; ++b) {
        const int64_t x = bsum[b];
        bsum[b] = run;
        run += x;
    }
    if (threadIdx.x == kThreads - 1) bsum[nb] = incl;
}

__global__ void __launch_bounds__(kThreads) scan_write(const int32_t *cnt, int64_t n, const int64_t *bsum,
                                                       int32_t *off, int64_t nb, int32_t *err) {
    __shared__ int64_t s_warp[kThreads / 32];
    __shared__ int32_t s_out[kScanTile];  // the tile's offsets, stored coalesced
    const int64_t t0 = int64_t(blockIdx.x) * kScanTile;
    const int64_t i0 = t0 + int64_t(threadIdx.x) * kScanItems;
    const int64_t mine = items_sum(cnt, n, i0);
    int64_t run = bsum[blockIdx.x] + block_incl_scan(mine, s_warp) - mine;
    bool big = false;
    for (int u = 0; u < kScanItems; ++u) {
        const int64_t i = i0 + u;
        big |= run > INT32_MAX;
        s_out[threadIdx.x * kScanItems + u] = int32_t(run);
        if (i < n) run += cnt[i];
    }
    if (big) atomicOr(err, ERR_CAPACITY);
    __syncthreads();
    const int64_t m = min(kScanTile, n - t0);
    for (int64_t u = threadIdx.x; u < m; u += kThreads) off[t0 + u] = s_out[u];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
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
    const int64_t nb = scan_tiles(nE);
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

// One coboundary pass over the current enumeration (the caller holds the
// context's lock).  *err_word receives the device error word.
gale_status run_pass(gale_ctx *ctx, uint32_t which, const EnumView &ev, int32_t *err_word) {
    const int64_t nE = ev.nE, nF = ev.nF;
    const uint64_t gen = ev.gen;
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
    // the pass reads the enumeration, its index and the canonical tet rows
    CbMesh m{};
    m.rows = reinterpret_cast<const int4 *>(cb.rows);
    m.cluster_of = cb.cluster_of;
    m.I_V = ctx->d_I_V;
    m.E = cb.E;
    m.F = cb.F;
    m.ebk = cb.ebk;
    m.fbk = cb.fbk;
    m.IE = cb.IE;
    m.IF = cb.IF;
    m.eo = cb.eo;
    m.ekw = cb.ekw;
    m.feo = cb.feo;
    m.fkc = cb.fkc;
    m.e2s = cb.e2s;
    m.f2s = cb.f2s;
    m.nv = hm.nv;
    m.nE = nE;
    m.nF = nF;
    m.sorted_ids = cb.sorted_ids;
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
    const int64_t nT = hm.nt;
    const int64_t rows_of[4] = {hm.nv, hm.nv, nE, nF};
    // entries: every edge is in two VE rows, every triangle in three VF and
    // three EF rows, every tet in four FT rows
    const int64_t len_of[4] = {2 * nE, 3 * nF, 3 * nF, 4 * nT};
    for (int rel = 0; rel < 4; ++rel)
        if (len_of[rel] >= INT32_MAX) return fail(GALE_EINVAL, "a coboundary relation has 2^31 or more entries");
    const bool wVF = which & GALE_CB_VF, wFT = which & GALE_CB_FT;
    // with the sorted numbering VF is gathered from VE and EF, which are then
    // built whether asked for or not; otherwise it is scattered like them
    const bool vf_gather = wVF && cb.sorted_ids;
    const bool wVE = (which & GALE_CB_VE) || vf_gather, wEF = (which & GALE_CB_EF) || vf_gather;
    const uint32_t place = (wVE ? GALE_CB_VE : 0u) | (wVF ? GALE_CB_VF : 0u) | (wEF ? GALE_CB_EF : 0u) |
                           (wFT ? GALE_CB_FT : 0u);
    // scratch: counters (zeroed), then the triangles' edge positions and the
    // tets' face positions
    auto al = [](int64_t x) { return (x + 3) & ~int64_t(3); };
    const int64_t n_ctr = 4 * al(hm.nv) + 4 * al(nE);
    const int64_t n_scr = n_ctr + 2 * al(nF) + 2 * al(nF) + (vf_gather ? 2 * al(nE) : 0);
    if (!grow(ctx, cb.scratch, cb.scratch_cap, std::max<int64_t>(n_scr, 4)) ||
        !grow(ctx, cb.cnt, cb.cnt_cap, std::max<int64_t>({hm.nv, nE, nF, int64_t(1)})))
        return fail(GALE_ENOMEM, "device allocation of coboundary scratch failed");
    Scatter sc{};
    {
        int32_t *q = cb.scratch;
        auto take = [&](int64_t n) {
            int32_t *r = q;
            q += al(n);
            return r;
        };
        sc.ve_n = take(hm.nv);
        sc.ve_fill = take(hm.nv);
        sc.vf_n = take(hm.nv);
        sc.vf_fill = take(hm.nv);
        sc.ef_lo = take(nE);
        sc.ef_mid = take(nE);
        sc.ef_lofill = take(nE);
        sc.ef_midfill = take(nE);
        sc.tri_ac = take(nF);
        sc.tri_bc = take(nF);
        sc.ft_slot = reinterpret_cast<int2 *>(take(2 * nF));
        sc.ef_tail = vf_gather ? reinterpret_cast<int2 *>(take(2 * nE)) : nullptr;
    }
    sc.cnt = cb.cnt;
    if (cudaMemsetAsync(cb.scratch, 0, sizeof(int32_t) * size_t(n_ctr), s) != cudaSuccess)
        return fail(GALE_ECUDA, "cudaMemsetAsync");
    // counts of the scattered parts
    if (wVE) k_sc_edges<false><<<grid_for(nE), kThreads, 0, s>>>(m, sc, ctx->d_err);
    if (wEF || wVF) k_sc_tris<false><<<grid_for(nF), kThreads, 0, s>>>(m, sc, wEF, wVF && !vf_gather, ctx->d_err);
    if (vf_gather) k_vf_count_sorted<<<grid_for(nE), kThreads, 0, s>>>(m, sc);
    const bool ft_gen = wFT && cb.ft_general;
    if (wFT && !ft_gen) {
        cudaMemsetAsync(sc.ft_slot, 0xff, sizeof(int2) * size_t(std::max<int64_t>(nF, 1)), s);
        k_ft_tets<FT_SLOTS><<<grid_for(nT), kThreads, 0, s>>>(m, sc, nT, ctx->d_err);
    }
    // row offsets, one relation at a time through the shared count array
    for (int rel : {int(REL_VE), int(REL_VF), int(REL_EF), int(REL_FT)}) {
        if (!(place & (1u << rel))) continue;
        const int64_t n = rows_of[rel];
        const int64_t nb = scan_tiles(n);
        if (!grow(ctx, cb.bsum, cb.bsum_cap, nb + 1) || !grow(ctx, cb.off[rel], cb.off_cap[rel], n + 1) ||
            !grow(ctx, cb.val[rel], cb.val_cap[rel], std::max<int64_t>(len_of[rel], 1)))
            return fail(GALE_ENOMEM, "device allocation of coboundary rows failed");
        const int grid = grid_for(n);
        switch (rel) {
            case REL_VE: k_len_ve<<<grid, kThreads, 0, s>>>(m, sc); break;
            case REL_VF: k_len_vf<<<grid, kThreads, 0, s>>>(m, sc, cb.fo); break;
            case REL_EF: k_len_ef<<<grid, kThreads, 0, s>>>(m, sc); break;
            default:
                if (ft_gen) {
                    cudaMemsetAsync(sc.cnt, 0, sizeof(int32_t) * size_t(std::max<int64_t>(nF, 1)), s);
                    k_ft_tets<FT_COUNT><<<grid_for(nT), kThreads, 0, s>>>(m, sc, nT, ctx->d_err);
                } else {
                    k_len_ft<<<grid, kThreads, 0, s>>>(m, sc, ctx->d_err);
                }
                break;
        }
        if (nb > 0) {
            scan_sums<<<int(nb), kThreads, 0, s>>>(cb.cnt, n, cb.bsum);
            scan_bsums<<<1, kThreads, 0, s>>>(cb.bsum, nb);
            scan_write<<<int(nb), kThreads, 0, s>>>(cb.cnt, n, cb.bsum, cb.off[rel], nb, ctx->d_err);
        } else {
            cudaMemsetAsync(cb.off[rel], 0, sizeof(int32_t), s);
        }
        cb.rows_of[rel] = n;
        cb.len[rel] = len_of[rel];
    }
    sc.ve_off = cb.off[REL_VE];
    sc.vf_off = cb.off[REL_VF];
    sc.ef_off = cb.off[REL_EF];
    sc.ft_off = cb.off[REL_FT];
    sc.ve_val = cb.val[REL_VE];
    sc.vf_val = cb.val[REL_VF];
    sc.ef_val = cb.val[REL_EF];
    sc.ft_val = cb.val[REL_FT];
    // values: cursors, scattered parts, then every row's contiguous part and
    // its order by id (sorted numbering: the scattered prefix only)
    k_cursors<<<grid_for(std::max(hm.nv, nE)), kThreads, 0, s>>>(m, sc, wVE, wVF, wEF);
    if (wVE) k_sc_edges<true><<<grid_for(nE), kThreads, 0, s>>>(m, sc, ctx->d_err);
    if (wEF || wVF)
        k_sc_tris<true><<<grid_for(nF), kThreads, 0, s>>>(m, sc, wEF, wVF && !vf_gather, ctx->d_err);
    const int32_t *fo = cb.fo;
    if (ft_gen) {
        cudaMemsetAsync(sc.cnt, 0, sizeof(int32_t) * size_t(std::max<int64_t>(nF, 1)), s);
        k_ft_tets<FT_FILL><<<grid_for(nT), kThreads, 0, s>>>(m, sc, nT, ctx->d_err);
        k_sort_rows<PL_FULL, 4, FRONT_NONE, 0><<<grid_for(nF), kThreads, 0, s>>>(m, sc, nF, sc.ft_off, sc.ft_val, fo);
    } else if (wFT) {
        k_ft_write<<<grid_for(nF), kThreads, 0, s>>>(m, sc);
    }
    if (wVE) k_sort_rows<PL_VE, 16, FRONT_NONE, 6144><<<grid_for(hm.nv), kThreads, 0, s>>>(m, sc, hm.nv, sc.ve_off, sc.ve_val, fo);
    if (wEF) k_sort_rows<PL_EF, 8, FRONT_EF, 0><<<grid_for(nE), kThreads, 0, s>>>(m, sc, nE, sc.ef_off, sc.ef_val, fo);
    if (vf_gather) k_vf_gather<<<grid_for(hm.nv), kThreads, 0, s>>>(m, sc, fo);
    else if (wVF)
        k_sort_rows<PL_VF, 32, FRONT_VF, 12288><<<grid_for(hm.nv), kThreads, 0, s>>>(m, sc, hm.nv, sc.vf_off, sc.vf_val, fo);
    if (cudaGetLastError() != cudaSuccess) return fail(GALE_ECUDA, "coboundary launch failed");
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(GALE_ECUDA, "cudaStreamSynchronize");
    int32_t e = 0;
    cudaMemcpy(&e, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost);
    *err_word = e;
    if (e) {
        cudaMemset(ctx->d_err, 0, sizeof(int32_t));
        return fail(GALE_EDEVICE, "coboundary pass: error word " + std::to_string(e));
    }
    return GALE_OK;
}

}  // namespace gale

extern "C" gale_status gale_build_coboundary(gale_ctx *ctx, uint32_t which, gale_coboundary *out) {
    using namespace gale;
    if (!ctx || !out) return fail(GALE_EINVAL, "NULL argument");
    if (ctx->device < 0) return fail(GALE_EINVAL, "host-only context");
    if (which == 0 || (which & ~uint32_t(GALE_CB_VE | GALE_CB_VF | GALE_CB_EF | GALE_CB_FT)))
        return fail(GALE_EINVAL, "which must be a non-empty set of GALE_CB_* bits");
    EnumView ev{};
    if (!enumeration_view(ctx, &ev)) return fail(GALE_ENOTFOUND, "no enumeration: call gale_enumerate first");
    if (ev.nE >= INT32_MAX || ev.nF >= INT32_MAX) return fail(GALE_EINVAL, "more than 2^31 - 1 edges or triangles");
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(GALE_ECUDA, "cudaSetDevice");
    if (!ctx->cb) ctx->cb = new Cobound();
    Cobound &cb = *ctx->cb;
    // a mesh the counting pass found non-manifold takes the general FT form
    // at once; otherwise a third tet on a triangle (the slots overflow)
    // switches this context to it and the pass runs again
    for (int32_t g : ctx->tt_general) cb.ft_general |= g != 0;
    int32_t e = 0;
    gale_status st = run_pass(ctx, which, ev, &e);
    if (st == GALE_EDEVICE && e == ERR_NONMANIFOLD && (which & GALE_CB_FT) && !cb.ft_general) {
        cb.ft_general = true;
        st = run_pass(ctx, which, ev, &e);
    }
    if (st != GALE_OK) return st;
    for (int rel = 0; rel < 4; ++rel) {
        const bool have = (which & (1u << rel)) != 0;
        out->rows[rel] = have ? cb.rows_of[rel] : 0;
        out->len[rel] = have ? cb.len[rel] : 0;
        out->off[rel] = have ? cb.off[rel] : nullptr;
        out->val[rel] = have ? cb.val[rel] : nullptr;
    }
    return GALE_OK;
}
