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
#include <mutex>
#include <random>
#include <thread>
#include <vector>

#include "gale.h"  // public C ABI only

namespace {

// Vertex w is below v when f(w) < f(v), ties broken by input id.
inline bool below(const float *f, const int32_t *inid, int32_t w, int32_t v) {
    return f[w] < f[v] || (f[w] == f[v] && inid[w] < inid[v]);
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
 * and VV rows to pinned host memory, classify, gale_release.
 *   f, inid, rows, I_V   host arrays in canonical order
 *   cls                  int8[nv] out (canonical order)
 *   lat                  double[K] out: seconds from request to view
 *   stats                double[4] out: wall seconds, requests, bytes D2H, failures
 */
int gale_cp_serve_run(gale_ctx *ctx, const float *f, const int32_t *inid, const int32_t *rows, const int64_t *I_V,
                      int32_t K, int32_t nthreads, uint32_t mask, uint64_t seed, double jump_prob, int8_t *cls,
                      double *lat, double *stats) {
    // K may be below the context's cluster count: only clusters [0, K) are served
    std::vector<std::atomic<uint8_t>> claimed(static_cast<size_t>(K));
    for (auto &c : claimed) c.store(0);
    std::atomic<int32_t> next_start{0};
    std::atomic<int64_t> done{0}, fails{0}, bytes{0};
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
            lat[k] = std::chrono::duration<double>(std::chrono::steady_clock::now() - r0).count();
            const int32_t nvo = v.v_end - v.v_begin;
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
            if (gale_cp_classify(f, inid, rows, int32_t(I_V[k]), nvo, pin, pin + need, pin + nvo + 1,
                                 pin + need + nvt, cls + I_V[k]) != 0)
                fails++;
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

}  // extern "C"
