// Coboundary relations VE, VF, EF, FT in the ids of the edge / triangle
// enumeration (Section 4.4: coboundary relations are computed by the GPU for
// whole segments; Section 5 evaluates VE, VF, EF and FT among them).
//
// Inputs on the device: the canonical tet rows, each vertex's cluster, the
// enumeration (E, F, their per-segment views in vertex-tuple order, I_E,
// I_F) and the VT and VV rows of every cluster from a batched build.  One
// thread per output row, two passes (count, then fill after an exclusive
// scan):
//   VE(v)  the edges {v, w} for w in VV(v), each found by binary search in
//          its segment's slice of E;
//   VF(v)  the triangles through v of the tets of VT(v), each taken from the
//          first tet of VT(v) that contains it;
//   EF(e)  for e = (u, w): the triangles (u, w, x) of the tets of VT(u) that
//          contain w, each from the first such tet;
//   FT(f)  for f = (a, b, c): the tets of VT(a) that contain b and c.
// Ids found by lookup are then sorted within their row.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gale_ctx.h"

namespace gale {

// device copies the coboundary pass keeps in the context
struct Cobound {
    const void *enm = nullptr;  // the enumeration the copies were made from
    int32_t *rows = nullptr, *cluster_of = nullptr;
    int32_t *E = nullptr, *F = nullptr, *ebk = nullptr, *fbk = nullptr;
    int64_t *IE = nullptr, *IF = nullptr;
    int64_t *base = nullptr;       // [K][4] bulk bases of the VT / VV segments
    int32_t *cnt = nullptr;        // counts of the largest relation
    int64_t *bsum = nullptr;       // scan block sums
    int64_t cnt_cap = 0, bsum_cap = 0;
    int32_t *off[4] = {}, *val[4] = {};
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

struct CbMesh {
    const int32_t *rows, *cluster_of, *I_V;
    const int32_t *E, *F, *ebk, *fbk;
    const int64_t *IE, *IF;
    const int32_t *vt_off, *vt_val, *vv_off, *vv_val;
    const int64_t *base;
    int64_t nv, nE, nF;
};

__device__ __forceinline__ void seg_row(const CbMesh &m, int32_t v, int which, int64_t &b, int64_t &e) {
    const int32_t k = m.cluster_of[v];
    const int32_t i = v - m.I_V[k];
    const int32_t *off = which ? m.vv_off : m.vt_off;
    const int64_t ob = m.base[4 * int64_t(k) + 2 * which], vb = m.base[4 * int64_t(k) + 2 * which + 1];
    b = vb + off[ob + i];
    e = vb + off[ob + i + 1];
}

__device__ __forceinline__ bool has(const int32_t *r, int32_t x) {
    return r[0] == x || r[1] == x || r[2] == x || r[3] == x;
}

__device__ int32_t lookup_edge(const CbMesh &m, int32_t u, int32_t w) {
    if (u > w) {
        const int32_t t = u;
        u = w;
        w = t;
    }
    const int32_t k = m.cluster_of[u];
    int64_t lo = m.IE[k], hi = m.IE[k + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t id = m.ebk[mid];
        const int32_t a = m.E[2 * int64_t(id)], b = m.E[2 * int64_t(id) + 1];
        if (a < u || (a == u && b < w)) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= m.IE[k + 1]) return -1;
    const int32_t id = m.ebk[lo];
    return (m.E[2 * int64_t(id)] == u && m.E[2 * int64_t(id) + 1] == w) ? id : -1;
}

__device__ int32_t lookup_face(const CbMesh &m, int32_t a, int32_t b, int32_t c) {
    // sort the three ids
    if (a > b) { const int32_t t = a; a = b; b = t; }
    if (b > c) { const int32_t t = b; b = c; c = t; }
    if (a > b) { const int32_t t = a; a = b; b = t; }
    const int32_t k = m.cluster_of[a];
    int64_t lo = m.IF[k], hi = m.IF[k + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t *f = m.F + 3 * int64_t(m.fbk[mid]);
        if (f[0] < a || (f[0] == a && (f[1] < b || (f[1] == b && f[2] < c)))) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= m.IF[k + 1]) return -1;
    const int32_t id = m.fbk[lo];
    const int32_t *f = m.F + 3 * int64_t(id);
    return (f[0] == a && f[1] == b && f[2] == c) ? id : -1;
}

// One row of relation REL: count (out == nullptr) or write its entries.
template <int REL>
__device__ int32_t row_entries(const CbMesh &m, int64_t row, int32_t *out, int32_t *err) {
    int32_t n = 0;
    if (REL == REL_VE) {
        const int32_t v = int32_t(row);
        int64_t b, e;
        seg_row(m, v, 1, b, e);
        for (int64_t j = b; j < e; ++j) {
            if (out) {
                const int32_t id = lookup_edge(m, v, m.vv_val[j]);
                if (id < 0) atomicOr(err, ERR_BAD_BLOCK);
                out[n] = id;
            }
            ++n;
        }
    } else if (REL == REL_VF) {
        const int32_t v = int32_t(row);
        int64_t b, e;
        seg_row(m, v, 0, b, e);
        for (int64_t j = b; j < e; ++j) {
            const int32_t *r = m.rows + 4 * int64_t(m.vt_val[j]);
            int32_t o[3], c = 0;
            for (int s = 0; s < 4; ++s)
                if (r[s] != v) o[c++] = r[s];
            const int32_t pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
            for (int p = 0; p < 3; ++p) {
                const int32_t x = o[pa[p]], y = o[pb[p]];
                bool first = true;
                for (int64_t jj = b; jj < j && first; ++jj) {
                    const int32_t *q = m.rows + 4 * int64_t(m.vt_val[jj]);
                    first = !(has(q, x) && has(q, y));
                }
                if (!first) continue;
                if (out) {
                    const int32_t id = lookup_face(m, v, x, y);
                    if (id < 0) atomicOr(err, ERR_BAD_BLOCK);
                    out[n] = id;
                }
                ++n;
            }
        }
    } else if (REL == REL_EF) {
        const int32_t u = m.E[2 * row], w = m.E[2 * row + 1];
        int64_t b, e;
        seg_row(m, u, 0, b, e);
        for (int64_t j = b; j < e; ++j) {
            const int32_t *r = m.rows + 4 * int64_t(m.vt_val[j]);
            if (!has(r, w)) continue;
            for (int s = 0; s < 4; ++s) {
                const int32_t x = r[s];
                if (x == u || x == w) continue;
                bool first = true;
                for (int64_t jj = b; jj < j && first; ++jj) {
                    const int32_t *q = m.rows + 4 * int64_t(m.vt_val[jj]);
                    first = !(has(q, w) && has(q, x));
                }
                if (!first) continue;
                if (out) {
                    const int32_t id = lookup_face(m, u, w, x);
                    if (id < 0) atomicOr(err, ERR_BAD_BLOCK);
                    out[n] = id;
                }
                ++n;
            }
        }
    } else {
        const int32_t a = m.F[3 * row], bb = m.F[3 * row + 1], cc = m.F[3 * row + 2];
        int64_t b, e;
        seg_row(m, a, 0, b, e);
        for (int64_t j = b; j < e; ++j) {
            const int32_t t = m.vt_val[j];
            const int32_t *r = m.rows + 4 * int64_t(t);
            if (has(r, bb) && has(r, cc)) {
                if (out) out[n] = t;
                ++n;
            }
        }
    }
    return n;
}

template <int REL>
__global__ void __launch_bounds__(kThreads) cb_count(CbMesh m, int64_t rows, int32_t *cnt, int32_t *err) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x)
        cnt[r] = row_entries<REL>(m, r, nullptr, err);
}

template <int REL>
__global__ void __launch_bounds__(kThreads) cb_fill(CbMesh m, int64_t rows, const int32_t *off, int32_t *val,
                                                    int32_t *err) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows; r += int64_t(gridDim.x) * blockDim.x) {
        int32_t *o = val + off[r];
        const int32_t n = row_entries<REL>(m, r, o, err);
        if (n != off[r + 1] - off[r]) {
            atomicOr(err, ERR_BAD_BLOCK);
            continue;
        }
        if (REL != REL_FT)  // ids found by lookup: sort the row (insertion sort)
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

__global__ void __launch_bounds__(kThreads) scan_bsums(int64_t *bsum, int64_t nb) {
    __shared__ int64_t s[kThreads];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += kThreads) {
        const int64_t b = b0 + threadIdx.x;
        const int64_t x = b < nb ? bsum[b] : 0;
        s[threadIdx.x] = x;
        __syncthreads();
        for (int o = 1; o < kThreads; o <<= 1) {
            const int64_t y = int(threadIdx.x) >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += y;
            __syncthreads();
        }
        if (b < nb) bsum[b] = carry + s[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == kThreads - 1) carry += s[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
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
T *upload(gale_ctx *ctx, const std::vector<T> &h, cudaStream_t s) {
    T *d = static_cast<T *>(ctx->dalloc(std::max<size_t>(h.size(), 1) * sizeof(T)));
    if (d && !h.empty()) cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    return d;
}

}  // namespace

// the enumeration's host arrays (gale_enum.cpp)
bool enumeration_arrays(gale_ctx *ctx, const std::vector<int32_t> **E, const std::vector<int32_t> **F,
                        const std::vector<int32_t> **ebk, const std::vector<int32_t> **fbk,
                        const std::vector<int64_t> **IE, const std::vector<int64_t> **IF);

}  // namespace gale

extern "C" gale_status gale_build_coboundary(gale_ctx *ctx, uint32_t which, gale_coboundary *out) {
    using namespace gale;
    if (!ctx || !out) return fail(GALE_EINVAL, "NULL argument");
    if (ctx->device < 0) return fail(GALE_EINVAL, "host-only context");
    if (which == 0 || (which & ~uint32_t(GALE_CB_VE | GALE_CB_VF | GALE_CB_EF | GALE_CB_FT)))
        return fail(GALE_EINVAL, "which must be a non-empty set of GALE_CB_* bits");
    if ((ctx->precond & (GALE_VT | GALE_VV)) != (GALE_VT | GALE_VV))
        return fail(GALE_EINVAL, "coboundary relations need VT and VV in the precondition mask");
    const std::vector<int32_t> *E, *F, *ebk, *fbk;
    const std::vector<int64_t> *IE, *IF;
    if (!enumeration_arrays(ctx, &E, &F, &ebk, &fbk, &IE, &IF))
        return fail(GALE_ENOTFOUND, "no enumeration: call gale_enumerate first");
    // the stars and neighbour sets of every vertex
    gale_status st = gale_build_clusters(ctx, nullptr, 0, GALE_VT | GALE_VV, GALE_MODE_BATCHED);
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
    if (cb.enm != static_cast<const void *>(ctx->enm)) {
        for (void *p : {static_cast<void *>(cb.E), static_cast<void *>(cb.F), static_cast<void *>(cb.ebk),
                        static_cast<void *>(cb.fbk), static_cast<void *>(cb.IE), static_cast<void *>(cb.IF)})
            if (p) ctx->dfree(p);
        cb.E = upload(ctx, *E, s);
        cb.F = upload(ctx, *F, s);
        cb.ebk = upload(ctx, *ebk, s);
        cb.fbk = upload(ctx, *fbk, s);
        cb.IE = upload(ctx, *IE, s);
        cb.IF = upload(ctx, *IF, s);
        if (!cb.E || !cb.F || !cb.ebk || !cb.fbk || !cb.IE || !cb.IF)
            return fail(GALE_ENOMEM, "device allocation of the enumeration failed");
        cb.enm = ctx->enm;
    }
    // bases of every cluster's VT / VV segments in the bulk arrays
    std::vector<int64_t> base(size_t(4) * K);
    for (int32_t k = 0; k < K; ++k) {
        const int64_t *o = ctx->bulk_offs.data() + size_t(10) * k;
        base[4 * size_t(k) + 0] = o[0];
        base[4 * size_t(k) + 1] = o[1];
        base[4 * size_t(k) + 2] = o[2];
        base[4 * size_t(k) + 3] = o[3];
    }
    if (cb.base) ctx->dfree(cb.base);
    cb.base = upload(ctx, base, s);
    if (!cb.base) return fail(GALE_ENOMEM, "device allocation failed");
    const int64_t nE = int64_t(E->size() / 2), nF = int64_t(F->size() / 3);
    const CbMesh m{cb.rows, cb.cluster_of, ctx->d_I_V, cb.E, cb.F, cb.ebk, cb.fbk, cb.IE, cb.IF,
                   ctx->bulk[0], ctx->bulk[1], ctx->bulk[2], ctx->bulk[3], cb.base, hm.nv, nE, nF};
    const int64_t rows_of[4] = {hm.nv, hm.nv, nE, nF};
    int sms = ctx->sm_count > 0 ? ctx->sm_count : 1;
    for (int rel = 0; rel < 4; ++rel) {
        if (!(which & (1u << rel))) continue;
        const int64_t n = rows_of[rel];
        const int64_t nb = (n + kThreads - 1) / kThreads;
        if (!grow(ctx, cb.cnt, cb.cnt_cap, std::max<int64_t>(n, 1)) ||
            !grow(ctx, cb.bsum, cb.bsum_cap, nb + 1) || !grow(ctx, cb.off[rel], cb.off_cap[rel], n + 1))
            return fail(GALE_ENOMEM, "device allocation of coboundary counts failed");
        const int grid = int(std::min<int64_t>(std::max<int64_t>(nb, 1), int64_t(sms) * 16));
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
        if (!grow(ctx, cb.val[rel], cb.val_cap[rel], std::max<int64_t>(total, 1)))
            return fail(GALE_ENOMEM, "device allocation of coboundary values failed");
        switch (rel) {
            case REL_VE: cb_fill<REL_VE><<<grid, kThreads, 0, s>>>(m, n, cb.off[rel], cb.val[rel], ctx->d_err); break;
            case REL_VF: cb_fill<REL_VF><<<grid, kThreads, 0, s>>>(m, n, cb.off[rel], cb.val[rel], ctx->d_err); break;
            case REL_EF: cb_fill<REL_EF><<<grid, kThreads, 0, s>>>(m, n, cb.off[rel], cb.val[rel], ctx->d_err); break;
            default: cb_fill<REL_FT><<<grid, kThreads, 0, s>>>(m, n, cb.off[rel], cb.val[rel], ctx->d_err); break;
        }
        if (cudaGetLastError() != cudaSuccess) return fail(GALE_ECUDA, "coboundary launch failed");
        cb.rows_of[rel] = n;
        cb.len[rel] = total;
    }
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
