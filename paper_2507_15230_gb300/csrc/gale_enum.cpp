// Edge and triangle enumeration and boundary relations, on the host.
//
// Section 4.3 ("Initialization") enumerates the mesh's edges and triangles on
// the CPU by iterating the tetrahedra of each segment and storing every two-
// and three-vertex combination in indexed lists E and F, with interval
// arrays I_E and I_F giving each segment's range.  An edge or triangle is
// internal to the segment of its lowest vertex.  Section 4.4 computes a
// boundary relation (FE, TE, TF) for one simplex by a few lookups in those
// lists, limited to the owning segment's interval.
//
// Segment k's edges and triangles are found among the tetrahedra of its
// working set (external, then internal, in canonical order): any simplex
// whose lowest vertex is in k lies in a tetrahedron containing that vertex.
// Two numberings within a segment: lexicographic in canonical ids, or the
// order of first appearance over those tetrahedra with each tetrahedron's
// combinations in combination order.  For lookups, each segment keeps a view
// of its ids sorted by vertex tuple (binary search), built on the first
// boundary query; in the lexicographic numbering that view is the identity.
#include <algorithm>
#include <atomic>
#include <array>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "gale_ctx.h"
#include "gale_enum.h"
#include "gale_par.h"

namespace gale {

struct Enumeration {
    int32_t order = -1;
    uint64_t gen = 0;                // distinct for every enumeration of the process
    raw_vector<int32_t> E;           // [2 nE] (u, w), u < w
    raw_vector<int32_t> F;           // [3 nF] (a, b, c), a < b < c
    std::vector<int64_t> I_E, I_F;   // [K+1]
    // ids in vertex-tuple order per segment; empty when the numbering is
    // lexicographic (identity)
    bool identity = false;
    raw_vector<int32_t> e_by_key;    // [nE]
    raw_vector<int32_t> f_by_key;    // [nF]
    int32_t ebk(int64_t j) const { return identity ? int32_t(j) : e_by_key[size_t(j)]; }
    int32_t fbk(int64_t p) const { return identity ? int32_t(p) : f_by_key[size_t(p)]; }
    // false while E and F exist only on the device (the sorted enumeration
    // of a device context); the first host query copies them (ensure_host_lists)
    std::atomic<bool> host_lists{true};
    std::mutex host_mu;
    // index inside each segment's interval, over the tuple order: a vertex's
    // upper edges and an edge's upper triangles are short runs.  Built by the
    // first boundary query (ensure_index).
    std::mutex index_mu;
    std::atomic<bool> indexed{false};
    std::vector<int32_t> v_eo;       // [nv+1] first tuple position of lower vertex v
    std::vector<int32_t> ekw;        // [nE] upper vertex of each tuple position
    std::vector<int32_t> e_feo;      // [nE+1] first triangle tuple position over each edge
    std::vector<int32_t> fkc;        // [nF] third vertex of each triangle tuple position
};

void enumeration_destroy(gale_ctx *ctx) {
    delete ctx->enm;
    ctx->enm = nullptr;
}

bool enumeration_view(gale_ctx *ctx, EnumView *v) {
    const Enumeration *en = ctx->enm;
    if (!en) return false;
    const int32_t K = ctx->hm.K;
    v->order = en->order;
    v->gen = en->gen;
    v->nE = en->I_E[size_t(K)];
    v->nF = en->I_F[size_t(K)];
    const bool h = en->host_lists.load(std::memory_order_acquire);
    v->E = h ? en->E.data() : nullptr;
    v->F = h ? en->F.data() : nullptr;
    v->ebk = en->identity ? nullptr : en->e_by_key.data();
    v->fbk = en->identity ? nullptr : en->f_by_key.data();
    v->IE = en->I_E.data();
    v->IF = en->I_F.data();
    v->K = K;
    return true;
}

namespace {

gale_status fail(gale_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

struct EKey {
    uint64_t key;  // u << 32 | w
    int64_t pos;   // order of first appearance
};
struct FKey {
    std::array<int32_t, 3> v;
    int64_t pos;
};

// One segment's simplices, numbered in `order`.
void segment_simplices(const HostMesh &hm, int32_t k, int32_t order, std::vector<uint64_t> &edges,
                       std::vector<std::array<int32_t, 3>> &faces) {
    const int32_t v0 = hm.I_V[k], v1 = hm.I_V[k + 1];
    std::vector<EKey> ek;
    std::vector<FKey> fk;
    int64_t pos = 0;
    auto visit = [&](int32_t t) {
        const int32_t *r = hm.rows.data() + 4 * int64_t(t);
        for (int i = 0; i < 4; ++i) {
            if (r[i] < v0 || r[i] >= v1) continue;  // lowest vertex of the combination must be own
            for (int j = i + 1; j < 4; ++j) {
                ek.push_back({uint64_t(uint32_t(r[i])) << 32 | uint32_t(r[j]), pos++});
                for (int l = j + 1; l < 4; ++l) fk.push_back({{r[i], r[j], r[l]}, pos++});
            }
        }
    };
    // combination order within a tetrahedron: (i, j) pairs and (i, j, l)
    // triples by increasing indices; interleaving edges and triangles above
    // keeps each kind's relative order
    for (int64_t x = hm.ext_off[k]; x < hm.ext_off[k + 1]; ++x) visit(hm.ext[x]);
    for (int32_t t = hm.I_T[k]; t < hm.I_T[k + 1]; ++t) visit(t);
    std::sort(ek.begin(), ek.end(),
              [](const EKey &a, const EKey &b) { return a.key != b.key ? a.key < b.key : a.pos < b.pos; });
    ek.erase(std::unique(ek.begin(), ek.end(), [](const EKey &a, const EKey &b) { return a.key == b.key; }),
             ek.end());
    std::sort(fk.begin(), fk.end(),
              [](const FKey &a, const FKey &b) { return a.v != b.v ? a.v < b.v : a.pos < b.pos; });
    fk.erase(std::unique(fk.begin(), fk.end(), [](const FKey &a, const FKey &b) { return a.v == b.v; }), fk.end());
    if (order == GALE_ENUM_FIRST_APPEARANCE) {
        std::sort(ek.begin(), ek.end(), [](const EKey &a, const EKey &b) { return a.pos < b.pos; });
        std::sort(fk.begin(), fk.end(), [](const FKey &a, const FKey &b) { return a.pos < b.pos; });
    }
    edges.resize(ek.size());
    for (size_t i = 0; i < ek.size(); ++i) edges[i] = ek[i].key;
    faces.resize(fk.size());
    for (size_t i = 0; i < fk.size(); ++i) faces[i] = fk[i].v;
}

// global id of edge (u, w), or -1
// tuple position of edge (u, w), u < w, or -1: a search among u's upper
// edges, which lie inside the interval of u's segment
int64_t edge_pos(const HostMesh &hm, const Enumeration &en, int32_t u, int32_t w) {
    if (u < 0 || u >= hm.nv) return -1;
    const int64_t b = en.v_eo[u], e = en.v_eo[u + 1];
    const int32_t *p = std::lower_bound(en.ekw.data() + b, en.ekw.data() + e, w);
    return (p != en.ekw.data() + e && *p == w) ? int64_t(p - en.ekw.data()) : -1;
}

int64_t edge_id(const HostMesh &hm, const Enumeration &en, int32_t u, int32_t w) {
    if (u > w) std::swap(u, w);
    const int64_t j = edge_pos(hm, en, u, w);
    return j < 0 ? -1 : en.ebk(j);
}

int64_t face_id(const HostMesh &hm, const Enumeration &en, std::array<int32_t, 3> f) {
    std::sort(f.begin(), f.end());
    const int64_t j = edge_pos(hm, en, f[0], f[1]);
    if (j < 0) return -1;
    for (int64_t p = en.e_feo[j]; p < en.e_feo[j + 1]; ++p) {
        if (en.fkc[p] == f[2]) return en.fbk(p);
        if (en.fkc[p] > f[2]) break;
    }
    return -1;
}

// The index over each segment's vertex-tuple order, from the enumeration's
// lists: one sweep per segment over its vertices, edges and triangles.
void build_index(Enumeration &en, const HostMesh &hm) {
    const int32_t K = hm.K;
    const int64_t nE = en.I_E[K], nF = en.I_F[K];
    en.v_eo.assign(size_t(hm.nv) + 1, int32_t(nE));
    en.ekw.resize(size_t(nE));
    en.e_feo.assign(size_t(nE) + 1, int32_t(nF));
    en.fkc.resize(size_t(nF));
    parallel_dynamic(K, host_threads(0), 16, [&](int64_t k, int) {
        const int64_t e0 = en.I_E[k], e1 = en.I_E[k + 1], f0 = en.I_F[k], f1 = en.I_F[k + 1];
        auto eu = [&](int64_t j) { return en.E[2 * size_t(en.ebk(j))]; };
        auto ew = [&](int64_t j) { return en.E[2 * size_t(en.ebk(j)) + 1]; };
        auto fa = [&](int64_t p, int c) { return en.F[3 * size_t(en.fbk(p)) + size_t(c)]; };
        int64_t j = e0, q = f0;
        for (int32_t v = hm.I_V[k]; v < hm.I_V[k + 1]; ++v) {
            while (j < e1 && eu(j) < v) ++j;
            en.v_eo[v] = int32_t(j);
        }
        for (j = e0; j < e1; ++j) {
            const int32_t a = eu(j), b = ew(j);
            en.ekw[j] = b;
            while (q < f1 && (fa(q, 0) < a || (fa(q, 0) == a && fa(q, 1) < b))) ++q;
            en.e_feo[j] = int32_t(q);
        }
        for (q = f0; q < f1; ++q) en.fkc[q] = fa(q, 2);
    });
}

gale_status ensure_host_lists(gale_ctx *ctx, Enumeration &en) {
    if (en.host_lists.load(std::memory_order_acquire)) return GALE_OK;
    std::lock_guard<std::mutex> lock(en.host_mu);
    if (en.host_lists.load(std::memory_order_relaxed)) return GALE_OK;
    const int32_t *dE = nullptr, *dF = nullptr;
    if (!device_enumeration(ctx, en.gen, &dE, &dF))
        return fail(GALE_ENOTFOUND, "the enumeration's lists are gone from the device");
    const int32_t K = ctx->hm.K;
    en.E.resize(size_t(2) * size_t(en.I_E[K]));
    en.F.resize(size_t(3) * size_t(en.I_F[K]));
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(GALE_ECUDA, "cudaSetDevice");
    gale_status st = copy_to_host(ctx, en.E.data(), dE, en.E.size() * 4);
    if (st == GALE_OK) st = copy_to_host(ctx, en.F.data(), dF, en.F.size() * 4);
    if (st != GALE_OK) return st;
    en.host_lists.store(true, std::memory_order_release);
    return GALE_OK;
}

void ensure_index(Enumeration &en, const HostMesh &hm) {
    if (en.indexed.load(std::memory_order_acquire)) return;
    std::lock_guard<std::mutex> lock(en.index_mu);
    if (en.indexed.load(std::memory_order_relaxed)) return;
    build_index(en, hm);
    en.indexed.store(true, std::memory_order_release);
}

}  // namespace
}  // namespace gale

extern "C" {

gale_status gale_enumerate(gale_ctx *ctx, int32_t order) {
    if (!ctx) return gale::fail(GALE_EINVAL, "NULL argument");
    if (order != GALE_ENUM_SORTED && order != GALE_ENUM_FIRST_APPEARANCE)
        return gale::fail(GALE_EINVAL, "unknown enumeration order");
    const gale::HostMesh &hm = ctx->hm;
    const int32_t K = hm.K;
    if (hm.rows.size() != size_t(4) * size_t(hm.nt) || hm.cluster_of.size() != size_t(hm.nv))
        return gale::fail(GALE_EINVAL, "the context holds no host rows");
    static std::atomic<uint64_t> next_gen{1};
    if (order == GALE_ENUM_SORTED) {
        // on a device context the sorted lists come from the GPU: a segment's
        // edges in tuple order are its ET edges, and the triangles over an
        // edge (a, b) the distinct vertices c > b of the tets of ET(a, b)
        try {
            auto en = std::make_unique<gale::Enumeration>();
            en->gen = next_gen.fetch_add(1);
            const gale_status st = gale::enumerate_sorted_device(ctx, en->gen, en->I_E, en->I_F);
            if (st == GALE_OK) {
                std::lock_guard<std::mutex> lock(ctx->mu);
                en->order = order;
                en->identity = true;
                en->host_lists.store(false);
                delete ctx->enm;
                ctx->enm = en.release();
                return GALE_OK;
            }
            if (st != GALE_ENOTFOUND) return st;  // a device failure, not a missing device
        } catch (const std::bad_alloc &) {
            return gale::fail(GALE_ENOMEM, "host allocation failed during enumeration");
        }
    }
    std::lock_guard<std::mutex> lock(ctx->mu);
    try {
        std::vector<std::vector<uint64_t>> se(K);
        std::vector<std::vector<std::array<int32_t, 3>>> sf(K);
        gale::parallel_dynamic(K, gale::host_threads(0), 1,
                               [&](int64_t k, int) { gale::segment_simplices(hm, int32_t(k), order, se[k], sf[k]); });
        auto en = std::make_unique<gale::Enumeration>();
        en->order = order;
        en->gen = next_gen.fetch_add(1);
        en->I_E.assign(size_t(K) + 1, 0);
        en->I_F.assign(size_t(K) + 1, 0);
        for (int32_t k = 0; k < K; ++k) {
            en->I_E[k + 1] = en->I_E[k] + int64_t(se[k].size());
            en->I_F[k + 1] = en->I_F[k] + int64_t(sf[k].size());
        }
        if (en->I_E[K] > INT32_MAX || en->I_F[K] > INT32_MAX)
            return gale::fail(GALE_EINVAL, "more than 2^31 edges or triangles");
        en->E.resize(size_t(2) * size_t(en->I_E[K]));
        en->F.resize(size_t(3) * size_t(en->I_F[K]));
        en->identity = order == GALE_ENUM_SORTED;
        if (!en->identity) {
            en->e_by_key.resize(size_t(en->I_E[K]));
            en->f_by_key.resize(size_t(en->I_F[K]));
        }
        gale::parallel_dynamic(K, gale::host_threads(0), 4, [&](int64_t k, int) {
            const int64_t e0 = en->I_E[k], f0 = en->I_F[k];
            const auto &ev = se[k];
            const auto &fv = sf[k];
            for (size_t i = 0; i < ev.size(); ++i) {
                en->E[2 * (e0 + int64_t(i))] = int32_t(ev[i] >> 32);
                en->E[2 * (e0 + int64_t(i)) + 1] = int32_t(ev[i] & 0xffffffffu);
            }
            for (size_t i = 0; i < fv.size(); ++i)
                for (int c = 0; c < 3; ++c) en->F[3 * (f0 + int64_t(i)) + c] = fv[i][c];
            if (en->identity) return;
            // ids of the segment in tuple order
            int32_t *eb = en->e_by_key.data() + e0;
            for (size_t i = 0; i < ev.size(); ++i) eb[i] = int32_t(e0 + int64_t(i));
            int32_t *fb = en->f_by_key.data() + f0;
            for (size_t i = 0; i < fv.size(); ++i) fb[i] = int32_t(f0 + int64_t(i));
            std::sort(eb, eb + ev.size(), [&](int32_t a, int32_t b) { return ev[a - e0] < ev[b - e0]; });
            std::sort(fb, fb + fv.size(), [&](int32_t a, int32_t b) { return fv[a - f0] < fv[b - f0]; });
        });
        delete ctx->enm;
        ctx->enm = en.release();
    } catch (const std::bad_alloc &) {
        return gale::fail(GALE_ENOMEM, "host allocation failed during enumeration");
    }
    return GALE_OK;
}

gale_status gale_get_enumeration(gale_ctx *ctx, int64_t *counts, int32_t *edges, int64_t *I_E, int32_t *faces,
                                 int64_t *I_F) {
    if (!ctx) return gale::fail(GALE_EINVAL, "NULL argument");
    const gale::Enumeration *en = ctx->enm;
    if (!en) return gale::fail(GALE_ENOTFOUND, "no enumeration: call gale_enumerate first");
    const int32_t K = ctx->hm.K;
    if (counts) {
        counts[0] = en->I_E[K];
        counts[1] = en->I_F[K];
    }
    const int64_t nE = en->I_E[K], nF = en->I_F[K];
    if (!en->host_lists.load(std::memory_order_acquire)) {
        // lists still only on the device: copy them straight to the caller
        const int32_t *dE = nullptr, *dF = nullptr;
        if ((edges && nE) || (faces && nF)) {
            if (!gale::device_enumeration(ctx, en->gen, &dE, &dF))
                return gale::fail(GALE_ENOTFOUND, "the enumeration's lists are gone from the device");
            if (cudaSetDevice(ctx->device) != cudaSuccess) return gale::fail(GALE_ECUDA, "cudaSetDevice");
        }
        gale_status st = GALE_OK;
        if (edges && nE) st = gale::copy_to_host(ctx, edges, dE, size_t(nE) * 8);
        if (st == GALE_OK && faces && nF) st = gale::copy_to_host(ctx, faces, dF, size_t(nF) * 12);
        if (st != GALE_OK) return st;
    } else {
        const int th = gale::host_threads(0);
        if (edges && nE) gale::parallel_copy(edges, en->E.data(), 2 * nE, th);
        if (faces && nF) gale::parallel_copy(faces, en->F.data(), 3 * nF, th);
    }
    if (I_E) memcpy(I_E, en->I_E.data(), en->I_E.size() * 8);
    if (I_F) memcpy(I_F, en->I_F.data(), en->I_F.size() * 8);
    return GALE_OK;
}

gale_status gale_boundary(gale_ctx *ctx, int32_t relation, const int64_t *ids, int64_t n, int32_t *out) {
    if (!ctx || (n > 0 && (!ids || !out))) return gale::fail(GALE_EINVAL, "NULL argument");
    gale::Enumeration *en = ctx->enm;
    if (!en) return gale::fail(GALE_ENOTFOUND, "no enumeration: call gale_enumerate first");
    const gale::HostMesh &hm = ctx->hm;
    const int32_t K = hm.K;
    int width, limit;
    if (relation == GALE_REL_FE) {
        width = 3;
        limit = int32_t(std::min<int64_t>(en->I_F[K], INT32_MAX));
    } else if (relation == GALE_REL_TE) {
        width = 6;
        limit = int32_t(std::min<int64_t>(hm.nt, INT32_MAX));
    } else if (relation == GALE_REL_TF) {
        width = 4;
        limit = int32_t(std::min<int64_t>(hm.nt, INT32_MAX));
    } else {
        return gale::fail(GALE_EINVAL, "unknown boundary relation");
    }
    for (int64_t i = 0; i < n; ++i)
        if (ids[i] < 0 || ids[i] >= limit) return gale::fail(GALE_EINVAL, "simplex id out of range");
    try {
        const gale_status st = gale::ensure_host_lists(ctx, *en);
        if (st != GALE_OK) return st;
        gale::ensure_index(*en, hm);
    } catch (const std::bad_alloc &) {
        return gale::fail(GALE_ENOMEM, "host allocation of the enumeration index failed");
    }
    std::atomic<int32_t> missing{0};
    gale::parallel_for(n, gale::host_threads(0), [&](int64_t b, int64_t e, int) {
        for (int64_t i = b; i < e; ++i) {
            int32_t *o = out + i * width;
            int64_t got[6];
            if (relation == GALE_REL_FE) {
                const int32_t *f = en->F.data() + 3 * ids[i];
                got[0] = gale::edge_id(hm, *en, f[0], f[1]);
                got[1] = gale::edge_id(hm, *en, f[0], f[2]);
                got[2] = gale::edge_id(hm, *en, f[1], f[2]);
            } else {
                const int32_t *r = hm.rows.data() + 4 * ids[i];
                if (relation == GALE_REL_TE) {
                    int c = 0;
                    for (int a = 0; a < 4; ++a)
                        for (int d = a + 1; d < 4; ++d) got[c++] = gale::edge_id(hm, *en, r[a], r[d]);
                } else {
                    int c = 0;
                    for (int a = 0; a < 4; ++a)
                        for (int d = a + 1; d < 4; ++d)
                            for (int g = d + 1; g < 4; ++g) got[c++] = gale::face_id(hm, *en, {r[a], r[d], r[g]});
                }
            }
            for (int c = 0; c < width; ++c) {
                if (got[c] < 0) missing++;
                o[c] = int32_t(got[c]);
            }
        }
    });
    if (missing.load()) return gale::fail(GALE_EINVAL, "a simplex is missing from the enumeration");
    return GALE_OK;
}

}  // extern "C"
