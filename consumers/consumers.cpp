// Consumers of the producer: a lower-link critical-point classifier of a
// float32 scalar field (standing in for the paper's analysis algorithms,
// Section 5.2 "CriticalPoints", which requests VV and VT) and a serving
// driver that runs many classifier threads against gale_request.
//
// Uses the public C ABI only (include/gale.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <random>
#include <thread>
#include <vector>

#include "gale.h"  // public C ABI only

namespace {

// fn(i) for i in [0, n) on up to n threads; the calling thread runs the
// ranks whose thread could not be started.
template <class F>
void run_on_threads(int n, F &&fn) {
    std::vector<std::thread> th;
    int started = 0;
    try {
        th.reserve(size_t(n));
        for (; started < n; ++started) th.emplace_back(fn, started);
    } catch (const std::exception &) {
    }
    for (int i = started; i < n; ++i) fn(i);
    for (auto &t : th) t.join();
}

// Vertex w is below v when f(w) < f(v), ties broken by input id.
inline bool below(const float *f, const int32_t *inid, int32_t w, int32_t v) {
    return f[w] < f[v] || (f[w] == f[v] && inid[w] < inid[v]);
}

// (value, input id) as one unsigned integer ordered like below(): the
// float's bits made monotone (-0 and +0 made one value first), the id
// offset to unsigned.  Values must not be NaN.
inline uint64_t order_key(float fx, int32_t id) {
    fx += 0.0f;
    uint32_t u;
    std::memcpy(&u, &fx, 4);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return uint64_t(u) << 32 | (uint32_t(id) ^ 0x80000000u);
}

struct DSU {
    int32_t p[512];
    int32_t find(int32_t x) {
        while (p[x] != x) x = p[x] = p[p[x]];
        return x;
    }
};

}  // namespace

extern "C" {

/*
 * Classify the own vertices of one cluster from its VT and VV rows:
 * the link of v is VV(v) with an edge between two neighbours whenever they
 * lie on a common tet of VT(v) with v; count the connected components of
 * its lower part (neighbours below v) and of its upper part.
 * Codes: 0 minimum (no lower part), 3 maximum (no upper part), -1 regular
 * (one of each), 1 join saddle (several lower components, one upper),
 * 2 split saddle (one lower, several upper), 4 both several.
 *   f, inid     per canonical vertex: field value and input id
 *   rows        canonical tet rows (int32[4 nt])
 *   v0, nvo     the cluster's vertices [v0, v0 + nvo)
 *   vt_off/val, vv_off/val  its VT and VV rows (offsets from 0)
 *   out         int8[nvo]
 * Returns 0, or -1 if a link has more than 512 vertices.
 */
int gale_cp_classify(const float *f, const int32_t *inid, const int32_t *rows, int32_t v0, int32_t nvo,
                     const int32_t *vt_off, const int32_t *vt_val, const int32_t *vv_off, const int32_t *vv_val,
                     int8_t *out) {
    DSU lo, hi;
    for (int32_t i = 0; i < nvo; ++i) {
        const int32_t v = v0 + i;
        const int32_t *nb = vv_val + vv_off[i];
        const int32_t n = vv_off[i + 1] - vv_off[i];
        if (n > 512) return -1;
        for (int32_t a = 0; a < n; ++a) lo.p[a] = hi.p[a] = a;
        auto idx = [&](int32_t w) { return int32_t(std::lower_bound(nb, nb + n, w) - nb); };
        for (int32_t q = vt_off[i]; q < vt_off[i + 1]; ++q) {
            const int32_t *r = rows + 4 * int64_t(vt_val[q]);
            int32_t o[3], c = 0;
            for (int j = 0; j < 4; ++j)
                if (r[j] != v) o[c++] = r[j];
            for (int a = 0; a < 3; ++a)
                for (int b = a + 1; b < 3; ++b) {
                    const bool la = below(f, inid, o[a], v), lb = below(f, inid, o[b], v);
                    if (la != lb) continue;
                    DSU &d = la ? lo : hi;
                    const int32_t x = d.find(idx(o[a])), y = d.find(idx(o[b]));
                    if (x != y) d.p[x] = y;
                }
        }
        int nl = 0, nu = 0;
        for (int32_t a = 0; a < n; ++a) {
            if (below(f, inid, nb[a], v)) nl += lo.find(a) == a;
            else nu += hi.find(a) == a;
        }
        int8_t code;
        if (nl == 0) code = 0;
        else if (nu == 0) code = 3;
        else if (nl == 1 && nu == 1) code = -1;
        else if (nu == 1) code = 1;
        else if (nl == 1) code = 2;
        else code = 4;
        out[i] = code;
    }
    return 0;
}

/*
 * Serving driver: nthreads consumer threads classify every vertex of the
 * mesh through gale_request.  Each thread claims a start cluster, then walks
 * clusters in id order (kd-tree leaves are numbered depth first, so ids are
 * spatially coherent) and with probability jump_prob jumps to a random
 * cluster; a cluster is claimed through an atomic bitmap so each is
 * classified once.  Per cluster: gale_request(mask | VT | VV), copy the VT
 * and VV rows to pinned host memory, classify, gale_release.  With null_work
 * set, each view is released as soon as it is served (no copy, no
 * classification): the producer measured without the consumers' own work.
 *   f, inid, rows, I_V   host arrays in canonical order
 *   cls                  int8[nv] out (canonical order)
 *   lat                  double[K] out: seconds from request to view
 *   stats                double[6] out: wall seconds, requests, bytes D2H, failures,
 *                        and summed over requests the seconds of the copy to host
 *                        and of the classification (the paper's "data integration")
 */
int gale_cp_serve_run(gale_ctx *ctx, const float *f, const int32_t *inid, const int32_t *rows, const int64_t *I_V,
                      int32_t K, int32_t nthreads, uint32_t mask, uint64_t seed, double jump_prob, int32_t null_work,
                      int8_t *cls, double *lat, double *stats) {
    // K may be below the context's cluster count: only clusters [0, K) are served
    std::vector<std::atomic<uint8_t>> claimed(static_cast<size_t>(K));
    for (auto &c : claimed) c.store(0);
    std::atomic<int32_t> next_start{0};
    std::atomic<int64_t> done{0}, fails{0}, bytes{0}, copy_ns{0}, use_ns{0};
    const uint32_t m = mask | GALE_VT | GALE_VV;
    auto t0 = std::chrono::steady_clock::now();
    auto worker = [&](int tid) {
        std::mt19937_64 rng(seed * 1315423911ull + uint64_t(tid));
        std::uniform_real_distribution<double> U(0.0, 1.0);
        cudaStream_t st;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        std::vector<int32_t> h;  // pageable staging, grown on demand
        int32_t *pin = nullptr;
        size_t pin_cap = 0;
        auto claim = [&](int32_t k) {
            uint8_t z = 0;
            return k >= 0 && k < K && claimed[k].compare_exchange_strong(z, 1);
        };
        int32_t k = -1;
        for (;;) {
            // next cluster: continue the walk, jump, or take a fresh start
            int32_t cand = -1;
            if (k >= 0 && U(rng) >= jump_prob) {
                for (int32_t j = k + 1; j < K && j < k + 64; ++j)
                    if (claim(j)) { cand = j; break; }
            } else if (k >= 0) {
                for (int tries = 0; tries < 32 && cand < 0; ++tries) {
                    const int32_t j = int32_t(rng() % uint64_t(K));
                    if (claim(j)) cand = j;
                }
            }
            while (cand < 0) {
                const int32_t j = next_start.fetch_add(1);
                if (j >= K) break;
                if (claim(j)) cand = j;
            }
            if (cand < 0) break;
            k = cand;
            gale_view v;
            auto r0 = std::chrono::steady_clock::now();
            if (gale_request(ctx, k, m, 0, &v) != GALE_OK) {
                fails++;
                continue;
            }
            const auto r1 = std::chrono::steady_clock::now();
            lat[k] = std::chrono::duration<double>(r1 - r0).count();
            const int32_t nvo = v.v_end - v.v_begin;
            if (null_work) {  // the producer alone: the view is taken and handed back
                gale_release(ctx, &v);
                done++;
                continue;
            }
            // offsets first, then values
            const size_t need = size_t(2 * (nvo + 1));
            if (pin_cap < need) {
                if (pin) cudaFreeHost(pin);
                pin_cap = std::max(need * 2, size_t(1) << 16);
                cudaHostAlloc(reinterpret_cast<void **>(&pin), pin_cap * 4, cudaHostAllocDefault);
            }
            cudaMemcpyAsync(pin, v.vt_off, 4 * size_t(nvo + 1), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(pin + nvo + 1, v.vv_off, 4 * size_t(nvo + 1), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            const int32_t nvt = pin[nvo], nvv = pin[2 * nvo + 1];
            const size_t need2 = need + size_t(nvt) + size_t(nvv);
            if (pin_cap < need2) {
                h.assign(pin, pin + need);
                cudaFreeHost(pin);
                pin_cap = need2 * 2;
                cudaHostAlloc(reinterpret_cast<void **>(&pin), pin_cap * 4, cudaHostAllocDefault);
                std::copy(h.begin(), h.end(), pin);
            }
            cudaMemcpyAsync(pin + need, v.vt_val, 4 * size_t(nvt), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(pin + need + nvt, v.vv_val, 4 * size_t(nvv), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            bytes += 4 * int64_t(need2);
            gale_release(ctx, &v);
            const auto r2 = std::chrono::steady_clock::now();
            if (gale_cp_classify(f, inid, rows, int32_t(I_V[k]), nvo, pin, pin + need, pin + nvo + 1,
                                 pin + need + nvt, cls + I_V[k]) != 0)
                fails++;
            const auto r3 = std::chrono::steady_clock::now();
            copy_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(r2 - r1).count();
            use_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(r3 - r2).count();
            done++;
        }
        if (pin) cudaFreeHost(pin);
        cudaStreamDestroy(st);
    };
    std::vector<std::thread> th;
    for (int i = 0; i < nthreads; ++i) th.emplace_back(worker, i);
    for (auto &t : th) t.join();
    stats[0] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats[1] = double(done.load());
    stats[2] = double(bytes.load());
    stats[3] = double(fails.load());
    stats[4] = 1e-9 * double(copy_ns.load());
    stats[5] = 1e-9 * double(use_ns.load());
    return 0;
}

/*
 * Open-loop request driver for one or more loaded meshes.  Requests arrive
 * as a Poisson process of `rate` per second (rate <= 0: all at time zero, the
 * closed loop that measures capacity); request i asks mesh mi[i] for cluster
 * ks[i] with mask masks[i].  nworkers threads take the requests in arrival
 * order: each waits for its request's arrival time (sleeping until shortly
 * before it, then yielding), calls gale_request (no time limit) and
 * gale_release.
 *   lat    double[n] out: seconds from the scheduled arrival to the view
 *   stats  double[3] out: wall seconds, failures, first failing request (-1)
 */
int gale_open_loop(gale_ctx *const *ctxs, int32_t nctx, const int32_t *mi, const int32_t *ks, const uint32_t *masks,
                   int64_t n, double rate, uint64_t seed, int32_t nworkers, double *lat, double *stats) {
    using clk = std::chrono::steady_clock;
    std::vector<double> arr(static_cast<size_t>(n), 0.0);
    if (rate > 0) {
        std::mt19937_64 rng(seed);
        std::exponential_distribution<double> gap(rate);
        double t = 0;
        for (int64_t i = 0; i < n; ++i) arr[i] = (t += gap(rng));
    }
    std::atomic<int64_t> next{0}, fails{0}, first_fail{-1};
    const auto t0 = clk::now();
    auto worker = [&]() {
        for (;;) {
            const int64_t i = next.fetch_add(1);
            if (i >= n) return;
            const auto due = t0 + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(arr[i]));
            if (clk::now() + std::chrono::microseconds(200) < due)
                std::this_thread::sleep_until(due - std::chrono::microseconds(200));
            while (clk::now() < due) std::this_thread::yield();
            gale_view v;
            const int32_t m = mi[i];
            gale_status st = (m >= 0 && m < nctx) ? gale_request(ctxs[m], ks[i], masks[i], 0, &v) : GALE_EINVAL;
            lat[i] = std::chrono::duration<double>(clk::now() - due).count();
            if (st != GALE_OK) {
                fails++;
                int64_t none = -1;
                first_fail.compare_exchange_strong(none, i);
                continue;
            }
            gale_release(ctxs[m], &v);
        }
    };
    std::vector<std::thread> th;
    for (int w = 0; w < nworkers; ++w) th.emplace_back(worker);
    for (auto &t : th) t.join();
    stats[0] = std::chrono::duration<double>(clk::now() - t0).count();
    stats[1] = double(fails.load());
    stats[2] = double(first_fail.load());
    return 0;
}


/*
 * Discrete gradient (Section 5.1, DiscreteGradient): a Forman discrete
 * vector field of the vertex field f, built lower star by lower star.  The
 * lower star of v holds every simplex that contains v and whose other
 * vertices are all below v; it is processed alone (the construction of
 * Robins, Wood and Sheppard, 2011):
 *   - an empty lower star makes v critical (a minimum);
 *   - otherwise v is paired with the lower-star edge of smallest value
 *     sequence and every other edge waits in the "zero" queue;
 *   - a simplex all of whose faces inside the lower star but one are
 *     classified enters the "one" queue; popping it pairs it with that face,
 *     or moves it to the zero queue if none is left;
 *   - when the one queue is empty, the smallest still-open entry of the zero
 *     queue becomes critical.
 * A simplex's value sequence lists its vertices other than v from highest to
 * lowest; sequences compare lexicographically, a proper prefix first.  The
 * faces inside the lower star are those that contain v, v itself excluded.
 *
 * The relations read are the ones the paper lists for this algorithm: the
 * coboundary rows VE(v), VF(v), VT(v) (GPU-built) and the vertex lists EV,
 * FV, TV.  The boundary relations FE and TF are answered by the consumer
 * itself, as Section 4.4 has consumers do, by a lookup among the lower
 * star's own simplices: a face through v is identified by its vertices.
 *   f, inid          per canonical vertex: value and input id
 *   [v_begin, v_end) vertices whose lower stars are processed
 *   ve/vf/vt_off,val CSR rows indexed by canonical vertex id (int64 offsets)
 *   ev int32[2 nE], fv int32[3 nF], tv int32[4 nT]  ascending vertex ids
 * Output, one entry per simplex, -1 where unpaired (a simplex is critical
 * when both of its entries are -1); every simplex whose highest vertex is in
 * the range gets both of its entries written:
 *   v_up[v]  edge paired with v        e_down[e]  vertex paired with e
 *   e_up[e]  triangle paired with e    f_down[f]  edge paired with f
 *   f_up[f]  tet paired with f         t_down[t]  triangle paired with t
 * VE and VF rows must list ids in ascending order (as the coboundary pass
 * writes them).  Returns 0, or -1 if the relations are inconsistent (a row
 * whose simplex lacks v, or a face of a lower-star simplex missing from the
 * lower star).
 */
namespace {

struct LowerStar {
    // local simplices: edges [0, ne), triangles [ne, ne + nf), tets after
    std::vector<int32_t> gid, seq, open, state, face, cof_off, cof, fill;
    std::vector<int32_t> order, rank, eidx, at, pos;  // at: simplex at each queue position; pos: its inverse
    std::vector<uint64_t> kidx, one, zero;            // sort keys; the two queues as position bitsets
    // dense ordering of small lower stars: one bit per rank triple
    static constexpr int kDense = 1 << 14;
    uint64_t dbits[kDense / 64];
    std::vector<int32_t> dslot = std::vector<int32_t>(kDense);
    std::vector<uint32_t> key;  // packed value sequence (ranks of the other vertices, highest first)
    // small lower stars (at most kSmall edges): vertex -> edge hash and
    // edge pair -> triangle table
    static constexpr int kSmall = 32, kHash = 64;
    int32_t hkey[kHash], hval[kHash];
    int32_t tri2[kSmall * kSmall];
};

struct DgArgs {
    const float *f;
    const int32_t *inid;
    const uint64_t *vk;  // order_key of every vertex, or null (computed on the fly)
    const int64_t *ve_off, *vf_off, *vt_off;
    const int32_t *ve_val, *vf_val, *vt_val, *ev, *fv, *tv;
    int32_t *v_up, *e_down, *e_up, *f_down, *f_up, *t_down;
};

// 0 ok, -1 inconsistent relations
int dg_vertex(const DgArgs &a, int32_t v, LowerStar &L) {
    const float *f = a.f;
    const int32_t *inid = a.inid;
    auto lt = [&](int32_t x, int32_t y) { return below(f, inid, x, y); };
    // lower-star edges, triangles and tets with their other vertices.  Every
    // row entry is written to the next slot and the slot is kept only when
    // all its other vertices are below v (no data-dependent branch).
    const int64_t ve0 = a.ve_off[v], ve1 = a.ve_off[v + 1], vf0 = a.vf_off[v], vf1 = a.vf_off[v + 1];
    const int64_t vt0 = a.vt_off[v], vt1 = a.vt_off[v + 1];
    const size_t cap = size_t((ve1 - ve0) + (vf1 - vf0) + (vt1 - vt0));
    if (L.gid.size() < cap) {
        L.gid.resize(cap);
        L.seq.resize(3 * cap);
    }
    int32_t *gid = L.gid.data(), *seq = L.seq.data();
    const uint64_t *vk = a.vk;
    auto key = [&](int32_t x) { return vk ? vk[x] : order_key(f[x], inid[x]); };
    const uint64_t kv = key(v);
    auto low = [&](int32_t x) -> int32_t { return int32_t(key(x) < kv); };  // below(x, v)
    // The output entries of every star simplex are written below, at ids
    // spread over the whole mesh: their lines are requested here already.
    int32_t n = 0, bad = 0;
    for (int64_t q = ve0; q < ve1; ++q) {
        const int32_t e = a.ve_val[q];
        __builtin_prefetch(a.e_down + e, 1);
        __builtin_prefetch(a.e_up + e, 1);
        const int32_t x = a.ev[2 * int64_t(e)], y = a.ev[2 * int64_t(e) + 1];
        bad |= int32_t(x != v) & int32_t(y != v);
        const int32_t o = x == v ? y : x;
        gid[n] = e;
        seq[3 * n] = o;
        seq[3 * n + 1] = seq[3 * n + 2] = -1;
        n += low(o);
    }
    const int32_t ne = n;
    for (int64_t q = vf0; q < vf1; ++q) {
        const int32_t t = a.vf_val[q];
        __builtin_prefetch(a.f_down + t, 1);
        __builtin_prefetch(a.f_up + t, 1);
        const int32_t *x = a.fv + 3 * int64_t(t);
        bad |= int32_t((x[0] == v) + (x[1] == v) + (x[2] == v) != 1);
        const int32_t o0 = x[0] == v ? x[1] : x[0], o1 = x[2] == v ? x[1] : x[2];
        gid[n] = t;
        seq[3 * n] = o0;
        seq[3 * n + 1] = o1;
        seq[3 * n + 2] = -1;
        n += low(o0) & low(o1);
    }
    const int32_t nf = n - ne;
    for (int64_t q = vt0; q < vt1; ++q) {
        const int32_t t = a.vt_val[q];
        __builtin_prefetch(a.t_down + t, 1);
        const int32_t *x = a.tv + 4 * int64_t(t);
        bad |= int32_t((x[0] == v) + (x[1] == v) + (x[2] == v) + (x[3] == v) != 1);
        const int32_t o0 = x[0] == v ? x[1] : x[0];
        const int32_t o1 = (x[0] == v) | (x[1] == v) ? x[2] : x[1];
        const int32_t o2 = x[3] == v ? x[2] : x[3];
        gid[n] = t;
        seq[3 * n] = o0;
        seq[3 * n + 1] = o1;
        seq[3 * n + 2] = o2;
        n += low(o0) & low(o1) & low(o2);
    }
    if (bad) return -1;
    const int32_t ns = n;
    // edges [0, ne), triangles [ne, ne + nf), tets after: a simplex's
    // dimension is also the number of its vertices other than v
    auto dim_of = [&](int32_t s) { return 1 + int32_t(s >= ne) + int32_t(s >= ne + nf); };
    if (ne == 0) {
        a.v_up[v] = -1;
        return ns == 0 ? 0 : -1;
    }
    // faces inside the lower star (the consumer's own FE / TF lookups): a
    // triangle (v, x, y) has the edges to x and to y, a tet (v, x, y, z) the
    // triangles on each pair of x, y, z.  Every other vertex is the far end
    // of a lower-star edge: eidx holds that edge per (simplex, other vertex),
    // found through a small hash (or a scan in large lower stars), and a
    // triangle is found from its two edges.
    // every entry read below is written first: a simplex's first dim_of(s)
    if (L.face.size() < size_t(ns) * 3) {
        L.face.resize(size_t(ns) * 3);
        L.eidx.resize(size_t(ns) * 3);
    }
    const bool small = ne <= LowerStar::kSmall;
    if (small) {
        for (int i = 0; i < LowerStar::kHash; ++i) L.hkey[i] = -1;
        for (int32_t e = 0; e < ne; ++e) {
            const int32_t x = L.seq[3 * size_t(e)];
            uint32_t h = (uint32_t(x) * 2654435761u) >> 26;
            while (L.hkey[h] >= 0) h = (h + 1) & (LowerStar::kHash - 1);
            L.hkey[h] = x;
            L.hval[h] = e;
        }
        for (int i = 0; i < ne * ne; ++i) L.tri2[i] = -1;
    }
    auto edge_to = [&](int32_t x) -> int32_t {
        if (small) {
            uint32_t h = (uint32_t(x) * 2654435761u) >> 26;
            for (int probe = 0; probe < LowerStar::kHash && L.hkey[h] >= 0; ++probe) {
                if (L.hkey[h] == x) return L.hval[h];
                h = (h + 1) & (LowerStar::kHash - 1);
            }
            return -1;
        }
        for (int32_t e = 0; e < ne; ++e)
            if (L.seq[3 * size_t(e)] == x) return e;
        return -1;
    };
    for (int32_t s = 0; s < ns; ++s) {
        if (dim_of(s) == 1) {
            L.eidx[3 * size_t(s)] = s;
            continue;
        }
        for (int i = 0; i < dim_of(s); ++i) {
            const int32_t e = edge_to(L.seq[3 * size_t(s) + i]);
            if (e < 0) return -1;
            L.eidx[3 * size_t(s) + i] = e;
        }
        if (dim_of(s) == 2) {
            L.face[3 * size_t(s)] = L.eidx[3 * size_t(s)];
            L.face[3 * size_t(s) + 1] = L.eidx[3 * size_t(s) + 1];
            if (small) {
                const int32_t i = L.eidx[3 * size_t(s)], j = L.eidx[3 * size_t(s) + 1];
                L.tri2[i * ne + j] = s;
                L.tri2[j * ne + i] = s;
            }
        }
    }
    auto tri_on = [&](int32_t i, int32_t j) -> int32_t {  // edge indices
        if (small) return L.tri2[i * ne + j];
        for (int32_t t = ne; t < ne + nf; ++t) {
            const int32_t p = L.eidx[3 * size_t(t)], q = L.eidx[3 * size_t(t) + 1];
            if ((p == i && q == j) || (p == j && q == i)) return t;
        }
        return -1;
    };
    for (int32_t s = ne + nf; s < ns; ++s) {
        const int32_t *e = &L.eidx[3 * size_t(s)];
        const int32_t l[3] = {tri_on(e[0], e[1]), tri_on(e[0], e[2]), tri_on(e[1], e[2])};
        for (int i = 0; i < 3; ++i) {
            if (l[i] < 0) return -1;
            L.face[3 * size_t(s) + i] = l[i];
        }
    }
    // value sequences.  Every other vertex of a lower-star simplex is the
    // far end of a lower-star edge, so the edges, ordered by value, rank
    // them 1..ne; a simplex's sequence is then its ranks, highest first,
    // packed 10 bits each (a proper prefix leaves zeros, so it compares
    // first).  Beyond 1023 lower neighbours the sequences compare by value.
    const bool packed = ne < 1024;
    L.rank.resize(size_t(ne));
    if (ne <= 32) {
        // few lower neighbours: rank = 1 + the number of edges whose far end
        // is lower, counted over (value, input id) in one integer each;
        // -0 and +0 are the same value, as in below()
        uint64_t ek[32];
        for (int32_t e = 0; e < ne; ++e) ek[e] = key(L.seq[3 * size_t(e)]);
        for (int32_t e = 0; e < ne; ++e) {
            int32_t r = 1;
            for (int32_t j = 0; j < ne; ++j) r += int32_t(ek[j] < ek[e]);
            L.rank[e] = r;
        }
    } else {
        L.order.resize(size_t(ne));
        for (int32_t e = 0; e < ne; ++e) L.order[e] = e;
        std::sort(L.order.begin(), L.order.end(),
                  [&](int32_t x, int32_t y) { return lt(L.seq[3 * size_t(x)], L.seq[3 * size_t(y)]); });
        for (int32_t i = 0; i < ne; ++i) L.rank[L.order[i]] = i + 1;
    }
    if (packed) {
        L.key.resize(size_t(ns));
        for (int32_t s = 0; s < ns; ++s) {
            uint32_t r[3] = {0u, 0u, 0u};
            for (int i = 0; i < dim_of(s); ++i) r[i] = uint32_t(L.rank[L.eidx[3 * size_t(s) + i]]);
            const uint32_t hi = std::max(r[0], std::max(r[1], r[2])), lo = std::min(r[0], std::min(r[1], r[2]));
            L.key[s] = hi << 20 | (r[0] + r[1] + r[2] - hi - lo) << 10 | lo;
        }
    } else {
        for (int32_t s = 0; s < ns; ++s)
            std::sort(&L.seq[3 * size_t(s)], &L.seq[3 * size_t(s)] + dim_of(s),
                      [&](int32_t x, int32_t y) { return lt(y, x); });
    }
    // cofaces inside the lower star (CSR over local ids)
    L.cof_off.assign(size_t(ns) + 1, 0);
    for (int32_t s = ne; s < ns; ++s)
        for (int i = 0; i < dim_of(s); ++i) L.cof_off[L.face[3 * size_t(s) + i] + 1]++;
    for (int32_t s = 0; s < ns; ++s) L.cof_off[s + 1] += L.cof_off[s];
    L.cof.assign(size_t(L.cof_off[ns]), 0);
    L.fill.assign(L.cof_off.begin(), L.cof_off.end() - 1);
    for (int32_t s = ne; s < ns; ++s)
        for (int i = 0; i < dim_of(s); ++i) L.cof[L.fill[L.face[3 * size_t(s) + i]]++] = s;
    // open = faces inside the lower star not yet classified
    L.open.assign(size_t(ns), 0);
    for (int32_t s = ne; s < ns; ++s) L.open[s] = dim_of(s);
    L.state.assign(size_t(ns), 0);
    // Two simplices of one lower star never share a value sequence (their
    // vertex sets differ), so one ascending sort gives each a distinct
    // position.  Both queues are bitsets over positions: the smallest entry
    // is the lowest set bit.
    auto earlier = [&](int32_t x, int32_t y) {
        if (packed) return L.key[x] < L.key[y];
        const int32_t *sx = &L.seq[3 * size_t(x)], *sy = &L.seq[3 * size_t(y)];
        const int32_t nx = dim_of(x), ny = dim_of(y);
        for (int i = 0; i < nx && i < ny; ++i)
            if (sx[i] != sy[i]) return lt(sx[i], sy[i]);
        return nx < ny;
    };
    L.at.resize(size_t(ns));
    const uint32_t B = uint32_t(ne) + 1;  // rank digits 0..ne
    if (packed && B * B * B <= uint32_t(LowerStar::kDense)) {
        // few lower neighbours: the ranks (r0, r1, r2) index a dense bitmap
        // in lexicographic order; its set bits, in order, are the sort
        const int32_t nwd = int32_t((B * B * B + 63) >> 6);
        for (int32_t i = 0; i < nwd; ++i) L.dbits[i] = 0u;
        for (int32_t s = 0; s < ns; ++s) {
            const uint32_t k = L.key[s];
            const uint32_t d = ((k >> 20) * B + ((k >> 10) & 1023u)) * B + (k & 1023u);
            L.dbits[d >> 6] |= uint64_t(1) << (d & 63);
            L.dslot[d] = s;
        }
        int32_t i = 0;
        for (int32_t w = 0; w < nwd; ++w)
            for (uint64_t m = L.dbits[w]; m; m &= m - 1u) L.at[i++] = L.dslot[64 * w + __builtin_ctzll(m)];
        if (i != ns) return -1;  // two simplices with one vertex set: a repeated row entry
    } else if (packed) {
        L.kidx.resize(size_t(ns));
        for (int32_t s = 0; s < ns; ++s) L.kidx[s] = uint64_t(L.key[s]) << 32 | uint32_t(s);
        std::sort(L.kidx.begin(), L.kidx.end());
        for (int32_t i = 0; i < ns; ++i) L.at[i] = int32_t(L.kidx[i] & 0xffffffffu);
    } else {
        for (int32_t s = 0; s < ns; ++s) L.at[s] = s;
        std::sort(L.at.begin(), L.at.end(), earlier);
    }
    L.pos.resize(size_t(ns));
    for (int32_t i = 0; i < ns; ++i) L.pos[L.at[i]] = i;
    const int32_t nw = (ns + 63) >> 6;
    L.one.assign(size_t(nw), 0u);
    L.zero.assign(size_t(nw), 0u);
    int32_t n_one = 0, n_zero = 0;
    auto has = [&](const std::vector<uint64_t> &q, int32_t s) { return (q[L.pos[s] >> 6] >> (L.pos[s] & 63)) & 1u; };
    auto push = [&](std::vector<uint64_t> &q, int32_t &n, int32_t s) {
        const uint64_t bit = uint64_t(1) << (L.pos[s] & 63);
        uint64_t &w = q[L.pos[s] >> 6];
        if (!(w & bit)) {
            w |= bit;
            ++n;
        }
    };
    auto pop = [&](std::vector<uint64_t> &q, int32_t &n) -> int32_t {
        for (int32_t i = 0; i < nw; ++i)
            if (q[i]) {
                const int b = __builtin_ctzll(q[i]);
                q[i] &= q[i] - 1u;
                --n;
                return L.at[64 * i + b];
            }
        return -1;
    };
    auto classify = [&](int32_t s) {
        L.state[s] = 1;
        for (int32_t q = L.cof_off[s]; q < L.cof_off[s + 1]; ++q) L.open[L.cof[q]]--;
    };
    auto offer_cofaces = [&](int32_t s) {
        for (int32_t q = L.cof_off[s]; q < L.cof_off[s + 1]; ++q) {
            const int32_t c = L.cof[q];
            if (!L.state[c] && L.open[c] == 1 && !has(L.one, c)) push(L.one, n_one, c);
        }
    };
    int32_t first = 0;
    for (int32_t s = 1; s < ne; ++s)
        if (L.pos[s] < L.pos[first]) first = s;
    a.v_up[v] = L.gid[first];
    a.e_down[L.gid[first]] = v;
    a.e_up[L.gid[first]] = -1;
    classify(first);
    for (int32_t s = 0; s < ne; ++s)
        if (s != first) push(L.zero, n_zero, s);
    offer_cofaces(first);
    // every other simplex starts unpaired
    for (int32_t s = 0; s < ns; ++s) {
        if (s == first) continue;
        const int32_t g = L.gid[s];
        if (dim_of(s) == 1) a.e_down[g] = a.e_up[g] = -1;
        else if (dim_of(s) == 2) a.f_down[g] = a.f_up[g] = -1;
        else a.t_down[g] = -1;
    }
    auto pair = [&](int32_t lo, int32_t hi) {
        const int32_t gl = L.gid[lo], gh = L.gid[hi];
        if (dim_of(lo) == 1) {
            a.e_up[gl] = gh;
            a.f_down[gh] = gl;
        } else {
            a.f_up[gl] = gh;
            a.t_down[gh] = gl;
        }
    };
    while (n_one || n_zero) {
        while (n_one) {
            const int32_t x = pop(L.one, n_one);
            if (L.state[x]) continue;
            if (L.open[x] == 0) {
                push(L.zero, n_zero, x);
                continue;
            }
            int32_t g = -1;
            for (int i = 0; i < dim_of(x); ++i)
                if (!L.state[L.face[3 * size_t(x) + i]]) g = L.face[3 * size_t(x) + i];
            pair(g, x);
            classify(g);
            classify(x);
            offer_cofaces(x);
            offer_cofaces(g);
        }
        while (n_zero) {
            const int32_t g = pop(L.zero, n_zero);
            if (L.state[g]) continue;
            classify(g);  // critical
            offer_cofaces(g);
            break;
        }
    }
    return 0;
}

}  // namespace

int gale_dg_lower_stars(const float *f, const int32_t *inid, int64_t v_begin, int64_t v_end, const int64_t *ve_off,
                        const int32_t *ve_val, const int64_t *vf_off, const int32_t *vf_val, const int64_t *vt_off,
                        const int32_t *vt_val, const int32_t *ev, const int32_t *fv, const int32_t *tv,
                        int32_t *v_up, int32_t *e_down, int32_t *e_up,
                        int32_t *f_down, int32_t *f_up, int32_t *t_down) {
    const DgArgs a{f, inid, nullptr, ve_off, vf_off, vt_off, ve_val, vf_val, vt_val, ev, fv, tv,
                   v_up, e_down, e_up, f_down, f_up, t_down};
    LowerStar L;
    for (int64_t v = v_begin; v < v_end; ++v)
        if (dg_vertex(a, int32_t(v), L) != 0) return -1;
    return 0;
}

/*
 * The same over all nv vertices with nthreads consumer threads; each thread
 * takes blocks of `grain` consecutive vertices from a shared counter (lower
 * stars are disjoint, so the threads write disjoint entries).
 * stats double[2] out: wall seconds, vertices processed.  Returns 0, -1 for
 * inconsistent relations, -2 if the key array cannot be allocated.
 */
int gale_dg_run(const float *f, const int32_t *inid, int64_t nv, const int64_t *ve_off, const int32_t *ve_val,
                const int64_t *vf_off, const int32_t *vf_val, const int64_t *vt_off, const int32_t *vt_val,
                const int32_t *ev, const int32_t *fv, const int32_t *tv, int32_t *v_up, int32_t *e_down,
                int32_t *e_up, int32_t *f_down, int32_t *f_up, int32_t *t_down, int32_t nthreads, int64_t grain,
                double *stats) {
    if (nthreads < 1) nthreads = 1;
    if (grain < 1) grain = 1024;
    std::atomic<int64_t> next{0}, done{0};
    std::atomic<int> err{0};
    const auto t0 = std::chrono::steady_clock::now();
    // every vertex's order key, once (each is read by about 15 lower stars)
    std::unique_ptr<uint64_t[]> vk(new (std::nothrow) uint64_t[size_t(std::max<int64_t>(nv, 1))]);
    if (!vk) return -2;
    run_on_threads(nthreads, [&](int i) {  // the fill also takes the pages' first touch
        const int64_t b = nv * i / nthreads, e = nv * (i + 1) / nthreads;
        for (int64_t x = b; x < e; ++x) vk[size_t(x)] = order_key(f[x], inid[x]);
    });
    const DgArgs a{f, inid, vk.get(), ve_off, vf_off, vt_off, ve_val, vf_val, vt_val, ev, fv, tv,
                   v_up, e_down, e_up, f_down, f_up, t_down};
    auto worker = [&](int) {
        LowerStar L;
        for (;;) {
            const int64_t b = next.fetch_add(grain);
            if (b >= nv || err.load()) return;
            const int64_t e = std::min(nv, b + grain);
            for (int64_t v = b; v < e; ++v)
                if (dg_vertex(a, int32_t(v), L) != 0) {
                    err.store(1);
                    return;
                }
            done += e - b;
        }
    };
    run_on_threads(nthreads, worker);
    stats[0] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats[1] = double(done.load());
    return err.load() ? -1 : 0;
}

}  // extern "C"
