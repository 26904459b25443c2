// Host-side initialisation (Section 4.3, "Initialization"): input checks,
// canonical numbering, per-cluster working sets (internal tets, external
// tets T_ex, face halo) and their packing into 16-bit local blocks.
//
// Everything here is O(nv + nt) work split over std::thread workers:
// counting sorts instead of comparison sorts, and per-cluster work done
// cluster-parallel.  The result is uploaded once and never changes.
#include "gale_host.h"
#include "gale_par.h"

#include <algorithm>
#include <array>
#include <iterator>
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <thread>

namespace gale {

namespace {

inline void sort4(int32_t *r) {
    auto cs = [](int32_t &a, int32_t &b) {
        if (b < a) std::swap(a, b);
    };
    cs(r[0], r[1]); cs(r[2], r[3]); cs(r[0], r[2]); cs(r[1], r[3]); cs(r[1], r[2]);
}

// Stable counting sort of items [0, n) by key(i) in [0, nkeys).  Writes
// out[pos] = i and start[k] = first position of key k (start[nkeys] = n).
template <class Key>
void counting_sort(int64_t n, int32_t nkeys, int nthreads, Key key, int32_t *out, std::vector<int64_t> &start) {
    int p = nthreads;
    // per-chunk histograms: keep their memory bounded
    while (p > 1 && int64_t(p) * nkeys > (int64_t(1) << 26)) p /= 2;
    if (int64_t(p) > n) p = int(std::max<int64_t>(1, n));
    std::vector<int64_t> hist(size_t(p) * nkeys, 0);
    parallel_for(n, p, [&](int64_t b, int64_t e, int t) {
        int64_t *h = hist.data() + size_t(t) * nkeys;
        for (int64_t i = b; i < e; ++i) h[key(i)]++;
    });
    start.assign(size_t(nkeys) + 1, 0);
    int64_t run = 0;
    for (int32_t k = 0; k < nkeys; ++k) {
        start[k] = run;
        for (int t = 0; t < p; ++t) {
            int64_t c = hist[size_t(t) * nkeys + k];
            hist[size_t(t) * nkeys + k] = run;
            run += c;
        }
    }
    start[nkeys] = run;
    parallel_for(n, p, [&](int64_t b, int64_t e, int t) {
        int64_t *h = hist.data() + size_t(t) * nkeys;
        for (int64_t i = b; i < e; ++i) out[h[key(i)]++] = int32_t(i);
    });
}

}  // namespace

// The distinct values of a stream of non-negative ids, in first-seen order,
// each with its dense index (its position in that order): an open-addressing
// table that grows at half load, reused across calls, so a cluster costs
// O(entries) instead of a sort of all of them.
struct DistinctIds {
    std::vector<int32_t> tab, at, vals;
    uint32_t mask = 0;
    void reset(size_t expect) {
        size_t cap = 64;
        while (cap < 2 * expect) cap <<= 1;
        if (tab.size() != cap) {
            tab.resize(cap);
            at.resize(cap);
        }
        std::fill(tab.begin(), tab.end(), -1);
        mask = uint32_t(cap - 1);
        vals.clear();
    }
    // v's dense index, v added first if absent
    int32_t add(int32_t v) {
        uint32_t h = slot(v);
        if (tab[h] == v) return at[h];
        const int32_t i = int32_t(vals.size());
        tab[h] = v;
        at[h] = i;
        vals.push_back(v);
        if (2 * vals.size() > tab.size()) grow();
        return i;
    }
    // dense index of v, -1 when absent
    int32_t index(int32_t v) const {
        const uint32_t h = slot(v);
        return tab[h] == v ? at[h] : -1;
    }

  private:
    // v's slot, or the empty slot where it would go
    uint32_t slot(int32_t v) const {
        uint32_t h = (uint32_t(v) * 2654435761u) & mask;
        while (tab[h] != v && tab[h] >= 0) h = (h + 1) & mask;
        return h;
    }
    void grow() {
        tab.assign(2 * tab.size(), -1);
        at.resize(tab.size());
        mask = uint32_t(tab.size() - 1);
        for (size_t i = 0; i < vals.size(); ++i) {
            const uint32_t h = slot(vals[i]);
            tab[h] = vals[i];
            at[h] = int32_t(i);
        }
    }
};

int host_threads(int requested) {
    if (requested > 0) return requested;
    unsigned h = std::thread::hardware_concurrency();
    return h ? int(h) : 1;
}

bool prepare_host(const gale_mesh_desc &d, HostMesh &hm, std::string &err) {
    using clk = std::chrono::steady_clock;
    auto t0 = clk::now();
    const int P = host_threads(d.host_threads);
    const int64_t nv = d.nv, nt = d.nt;
    const int32_t K = d.nclusters;
    if (nv < 1 || nt < 0 || nv > INT32_MAX || nt > INT32_MAX - 1 || K < 1 || K > nv) {
        err = "invalid sizes (need 1 <= nv < 2^31, 0 <= nt < 2^31, 1 <= nclusters <= nv)";
        return false;
    }
    if (!d.seg || (nt > 0 && !d.tv)) {
        err = "tv and seg must be non-NULL host pointers";
        return false;
    }
    hm.nv = nv;
    hm.nt = nt;
    hm.K = K;
    const int32_t *seg = d.seg, *tv = d.tv;

    // ---- 1. input checks ----
    std::atomic<int64_t> bad_v{-1}, bad_t{-1};
    parallel_for(nv, P, [&](int64_t b, int64_t e, int) {
        for (int64_t v = b; v < e; ++v)
            if (seg[v] < 0 || seg[v] >= K) {
                bad_v = v;
                return;
            }
    });
    if (bad_v >= 0) {
        err = "segment id out of range at vertex " + std::to_string(bad_v.load());
        return false;
    }
    parallel_for(nt, P, [&](int64_t b, int64_t e, int) {
        for (int64_t t = b; t < e; ++t) {
            int32_t r[4];
            for (int j = 0; j < 4; ++j) {
                r[j] = tv[4 * t + j];
                if (r[j] < 0 || r[j] >= nv) {
                    bad_t = t;
                    return;
                }
            }
            sort4(r);
            if (r[0] == r[1] || r[1] == r[2] || r[2] == r[3]) {
                bad_t = t;
                return;
            }
        }
    });
    if (bad_t >= 0) {
        err = "tet " + std::to_string(bad_t.load()) + " has a vertex id out of range or a repeated vertex";
        return false;
    }

    // ---- 2. canonical vertex ids: stable by (segment, input id) ----
    hm.vperm.resize(nv);
    hm.cid.resize(nv);
    std::vector<int64_t> start;
    counting_sort(nv, K, P, [&](int64_t v) { return seg[v]; }, hm.vperm.data(), start);
    hm.I_V.resize(size_t(K) + 1);
    for (int32_t k = 0; k <= K; ++k) hm.I_V[k] = int32_t(start[k]);
    parallel_for(nv, P, [&](int64_t b, int64_t e, int) {
        for (int64_t c = b; c < e; ++c) hm.cid[hm.vperm[c]] = int32_t(c);
    });
    std::vector<int32_t> &cl = hm.cluster_of;  // canonical vertex -> cluster (nondecreasing)
    cl.resize(nv);
    parallel_for(nv, P, [&](int64_t b, int64_t e, int) {
        for (int64_t c = b; c < e; ++c) cl[c] = seg[hm.vperm[c]];
    });

    // ---- 3. canonical tets: rows relabelled and sorted, owner = cluster
    //         of the lowest vertex, stable by (owner, input index) ----
    std::vector<int32_t> rows_in(size_t(4) * nt);
    std::vector<int32_t> owner(nt);
    parallel_for(nt, P, [&](int64_t b, int64_t e, int) {
        for (int64_t t = b; t < e; ++t) {
            int32_t *r = rows_in.data() + 4 * t;
            for (int j = 0; j < 4; ++j) r[j] = hm.cid[tv[4 * t + j]];
            sort4(r);
            owner[t] = cl[r[0]];
        }
    });
    hm.tperm.resize(nt);
    counting_sort(nt, K, P, [&](int64_t t) { return owner[t]; }, hm.tperm.data(), start);
    hm.I_T.resize(size_t(K) + 1);
    for (int32_t k = 0; k <= K; ++k) hm.I_T[k] = int32_t(start[k]);
    hm.rows.resize(size_t(4) * nt);
    parallel_for(nt, P, [&](int64_t b, int64_t e, int) {
        for (int64_t c = b; c < e; ++c) memcpy(&hm.rows[4 * c], &rows_in[4 * int64_t(hm.tperm[c])], 16);
    });
    std::vector<int32_t>().swap(rows_in);
    std::vector<int32_t>().swap(owner);
    const int32_t *rows = hm.rows.data();

    // ---- 4. T_ex: a tet is external to every other cluster it touches.
    //         Clusters along a sorted row are nondecreasing, so the distinct
    //         ones are where consecutive entries differ. ----
    {
        // (cluster, tet) incidences, counted per tet
        std::vector<int64_t> per(nt + 1, 0);
        parallel_for(nt, P, [&](int64_t b, int64_t e, int) {
            for (int64_t t = b; t < e; ++t) {
                const int32_t *r = rows + 4 * t;
                per[t + 1] = (cl[r[1]] != cl[r[0]]) + (cl[r[2]] != cl[r[1]]) + (cl[r[3]] != cl[r[2]]);
            }
        });
        {  // inclusive prefix over the chunks of parallel_for: sums, then runs
            const int pc = int(std::max<int64_t>(1, std::min<int64_t>(P, nt)));
            std::vector<int64_t> csum(size_t(pc) + 1, 0);
            parallel_for(nt, pc, [&](int64_t b, int64_t e, int c) {
                int64_t x = 0;
                for (int64_t t = b; t < e; ++t) x += per[t + 1];
                csum[size_t(c) + 1] = x;
            });
            for (int c = 0; c < pc; ++c) csum[size_t(c) + 1] += csum[size_t(c)];
            parallel_for(nt, pc, [&](int64_t b, int64_t e, int c) {
                int64_t x = csum[size_t(c)];
                for (int64_t t = b; t < e; ++t) {
                    x += per[t + 1];
                    per[t + 1] = x;
                }
            });
        }
        const int64_t ninc = per[nt];
        std::vector<int32_t> inc_c(ninc), inc_t(ninc);
        parallel_for(nt, P, [&](int64_t b, int64_t e, int) {
            for (int64_t t = b; t < e; ++t) {
                const int32_t *r = rows + 4 * t;
                int64_t p = per[t];
                for (int j = 1; j < 4; ++j)
                    if (cl[r[j]] != cl[r[j - 1]]) {
                        inc_c[p] = cl[r[j]];
                        inc_t[p] = int32_t(t);
                        ++p;
                    }
            }
        });
        std::vector<int32_t> order(ninc);
        counting_sort(ninc, K, P, [&](int64_t i) { return inc_c[i]; }, order.data(), start);
        hm.ext_off.assign(start.begin(), start.end());
        hm.ext.resize(ninc);
        parallel_for(ninc, P, [&](int64_t b, int64_t e, int) {
            for (int64_t i = b; i < e; ++i) hm.ext[i] = inc_t[order[i]];
        });
    }

    // ---- 5. halo: tets outside T_k across the face (b, c, d) of an internal
    //         tet (a, b, c, d) whose only vertex in k is a ----
    hm.halo_off.assign(size_t(K) + 1, 0);
    hm.halo.clear();
    const bool want_tt = (d.precondition_mask & 8u) != 0;
    // vertex stars (the tets of each vertex, in no particular order: both
    // users sort what they collect), kept for the parts' halos.  Counted and
    // filled with atomic cursors: a stable counting sort over nv keys would
    // need per-thread histograms of nv entries.
    std::vector<int32_t> order;   // star of c: order[vs_off[c] .. vs_off[c+1]), tet ids
    std::vector<int64_t> vs_off;
    if (want_tt && nt > 0) {
        order.resize(size_t(4) * nt);
        vs_off.assign(size_t(nv) + 1, 0);
        parallel_for(4 * nt, P, [&](int64_t b, int64_t e, int) {
            for (int64_t i = b; i < e; ++i) __atomic_fetch_add(&vs_off[size_t(rows[i]) + 1], int64_t(1), __ATOMIC_RELAXED);
        });
        for (int64_t v = 0; v < nv; ++v) vs_off[v + 1] += vs_off[v];
        {
            std::vector<int64_t> cur(vs_off.begin(), vs_off.end() - 1);
            parallel_for(4 * nt, P, [&](int64_t b, int64_t e, int) {
                for (int64_t i = b; i < e; ++i)
                    order[size_t(__atomic_fetch_add(&cur[size_t(rows[i])], int64_t(1), __ATOMIC_RELAXED))] =
                        int32_t(i >> 2);
            });
        }
        std::vector<std::vector<int32_t>> halo_k(K);
        parallel_dynamic(K, P, 16, [&](int64_t k, int) {
            std::vector<int32_t> &hk = halo_k[k];
            for (int32_t t = hm.I_T[k]; t < hm.I_T[k + 1]; ++t) {
                const int32_t *r = rows + 4 * int64_t(t);
                if (cl[r[1]] == int32_t(k)) continue;  // face bcd has a vertex in k
                const int32_t b = r[1], c = r[2], dd = r[3];
                for (int64_t q = vs_off[b]; q < vs_off[b + 1]; ++q) {
                    const int32_t u = order[q];
                    if (u == t) continue;
                    const int32_t *ru = rows + 4 * int64_t(u);
                    bool hc = false, hd = false;
                    for (int j = 0; j < 4; ++j) {
                        hc |= ru[j] == c;
                        hd |= ru[j] == dd;
                    }
                    if (!hc || !hd) continue;
                    bool ink = false;
                    for (int j = 0; j < 4; ++j) ink |= cl[ru[j]] == int32_t(k);
                    if (!ink) hk.push_back(u);
                }
            }
            std::sort(hk.begin(), hk.end());
            hk.erase(std::unique(hk.begin(), hk.end()), hk.end());
        });
        int64_t run = 0;
        for (int32_t k = 0; k < K; ++k) {
            hm.halo_off[k] = run;
            run += int64_t(halo_k[k].size());
        }
        hm.halo_off[K] = run;
        hm.halo.resize(run);
        parallel_for(K, P, [&](int64_t b, int64_t e, int) {
            for (int64_t k = b; k < e; ++k)
                std::copy(halo_k[k].begin(), halo_k[k].end(), hm.halo.begin() + hm.halo_off[k]);
        });
    }

    // ---- 6. working sets and their blocks: every cluster, then the parts of
    //         the clusters too large for one CTA's shared memory ----
    // A working set: own vertices [v0, v1); external tets (ascending, below
    // every internal one); internal tets (the id range [t0, t1), or for a
    // part an ascending list); halo tets (ascending).
    struct WSet {
        int32_t v0 = 0, v1 = 0;
        const int32_t *ext = nullptr;
        int64_t n_ext = 0;
        int32_t t0 = 0, t1 = 0;
        const int32_t *ilist = nullptr;
        int64_t n_int = 0;
        const int32_t *halo = nullptr;
        int64_t n_halo = 0;
        int32_t part = 0;  // 0, or 1 + the part's index
        int32_t t_base = 0;
        int32_t itet(int64_t i) const { return ilist ? ilist[i] : t0 + int32_t(i); }
    };
    // vertex map and facts of a working set: 0 ok, 1 too large for 16-bit
    // local ids, 2 two internal tets with the same vertex set
    auto ws_scan = [&](const WSet &w, ClusterStat &s, std::vector<int32_t> &vm) -> int {
        const int32_t v0 = w.v0, v1 = w.v1;
        // neighbour universe: vertices of [external | internal] tets plus the
        // own interval, ascending; then halo-only vertices, ascending
        thread_local DistinctIds seen;
        std::vector<int32_t> nb, ho;
        seen.reset(size_t(v1 - v0) * 2 + 64);
        // each row entry's dense index among the non-own vertices, kept for
        // the upper-neighbour count below (own vertices: -1 - offset)
        thread_local std::vector<int32_t> code;
        code.resize(size_t(4) * size_t(w.n_ext + w.n_int));
        auto add_row = [&](int32_t t, int32_t *c) {
            const int32_t *r = rows + 4 * int64_t(t);
            for (int j = 0; j < 4; ++j) {
                const bool own = r[j] >= v0 && r[j] < v1;
                const int32_t d = own ? -1 - (r[j] - v0) : seen.add(r[j]);
                if (c) c[j] = d;
            }
        };
        for (int64_t i = 0; i < w.n_ext; ++i) add_row(w.ext[i], code.data() + 4 * i);
        for (int64_t i = 0; i < w.n_int; ++i) add_row(w.itet(i), code.data() + 4 * (w.n_ext + i));
        nb = seen.vals;
        std::sort(nb.begin(), nb.end());
        const size_t n_nb = seen.vals.size();
        for (int64_t i = 0; i < w.n_halo; ++i) add_row(w.halo[i], nullptr);
        ho.assign(seen.vals.begin() + int64_t(n_nb), seen.vals.end());  // halo-only: not seen before
        std::sort(ho.begin(), ho.end());
        const int64_t below = std::lower_bound(nb.begin(), nb.end(), v0) - nb.begin();
        vm.clear();
        vm.reserve(nb.size() + (v1 - v0) + ho.size());
        vm.insert(vm.end(), nb.begin(), nb.begin() + below);
        for (int32_t v = v0; v < v1; ++v) vm.push_back(v);
        vm.insert(vm.end(), nb.begin() + below, nb.end());
        const int32_t nv_nb = int32_t(vm.size());
        vm.insert(vm.end(), ho.begin(), ho.end());
        s = ClusterStat{};
        s.n_ext = int32_t(w.n_ext);
        s.n_own = int32_t(w.n_int);
        s.n_halo = int32_t(w.n_halo);
        s.nv_loc = int32_t(vm.size());
        s.nv_nb = nv_nb;
        s.nv_own = v1 - v0;
        s.xmap = w.part ? s.n_own : 0;
        const int64_t ntot = w.n_ext + w.n_int + w.n_halo;
        if (int64_t(vm.size()) > kMaxLocal || ntot > kMaxLocal - 1) return 1;
        // degrees and distinct upper neighbours of own vertices over
        // [external | internal]
        const int32_t nvo = v1 - v0;
        std::vector<int32_t> vm_up, ufill(static_cast<size_t>(v1 - v0) + 1, 0);
        // per own vertex: its incidences, and its upper neighbours bucketed
        // in one array by a counting pass and a fill pass, as dense ids
        // (own vertex v0 + i -> n_nb + i, any other -> its index among the
        // neighbour universe; only their number of distinct values matters)
        std::vector<int32_t> deg(static_cast<size_t>(nvo), 0), uoff(static_cast<size_t>(nvo) + 1, 0);
        for (int pass = 0; pass < 2; ++pass) {
            auto row = [&](int64_t i) {
                const int32_t *c = code.data() + 4 * i;
                for (int j = 0; j < 4; ++j)
                    if (c[j] < 0) {
                        const int32_t x = -1 - c[j];
                        if (pass == 0) {
                            deg[x]++;
                            uoff[x + 1] += 3 - j;
                        } else {
                            for (int q = j + 1; q < 4; ++q)
                                vm_up[uoff[x]++] = c[q] < 0 ? int32_t(n_nb) - 1 - c[q] : c[q];
                        }
                    }
            };
            if (pass == 1) {
                for (int32_t x = 0; x < nvo; ++x) uoff[x + 1] += uoff[x];
                vm_up.resize(size_t(uoff[nvo]));
                std::copy(uoff.begin(), uoff.end() - 1, ufill.begin());
                std::swap(uoff, ufill);  // uoff: fill cursors; ufill: row starts
            }
            for (int64_t i = 0; i < w.n_ext + w.n_int; ++i) row(i);
        }
        int32_t nvt = 0, mx = 0, mu = 0, ne = 0;
        thread_local std::vector<int32_t> stamp;
        stamp.assign(n_nb + size_t(nvo), -1);
        for (int32_t x = 0; x < nvo; ++x) {
            nvt += deg[x];
            mx = std::max(mx, deg[x]);
            int32_t nu = 0;
            for (int32_t i = ufill[x]; i < uoff[x]; ++i) {
                int32_t &st = stamp[size_t(vm_up[i])];
                nu += st != x;
                st = x;
            }
            mu = std::max(mu, nu);
            ne += nu;
        }
        s.n_vt = nvt;
        s.max_deg = mx;
        s.max_up = mu;
        s.n_e = ne;
        // internal tets with an own lowest vertex whose face opposite it has
        // no own vertex
        int32_t nbnd = 0;
        for (int64_t i = 0; i < w.n_int; ++i) {
            const int32_t *r = rows + 4 * int64_t(w.itet(i));
            nbnd += (r[0] >= v0 && r[0] < v1 && r[1] >= v1);
        }
        s.n_bnd = nbnd;
        // two tets with the same vertex set have the same owner and the same
        // lowest vertex: compare the rows of each own vertex's internal tets
        if (!w.part && w.n_int > 1) {
            std::vector<int32_t> first(size_t(nvo), -1), next(size_t(w.n_int), -1);
            for (int64_t i = 0; i < w.n_int; ++i) {
                const int32_t *r = rows + 4 * int64_t(w.itet(i));
                const int32_t x = r[0] - v0;
                if (x < 0 || x >= nvo) continue;
                for (int32_t q = first[x]; q >= 0; q = next[q])
                    if (memcmp(r, rows + 4 * int64_t(w.itet(q)), 16) == 0) return 2;
                next[i] = first[x];
                first[x] = int32_t(i);
            }
        }
        return 0;
    };
    auto ws_fill = [&](const WSet &w, const ClusterStat &s, const std::vector<int32_t> &vm, int32_t *blk,
                       int64_t words) {
        memset(blk, 0, size_t(words) * 4);
        const int32_t v0 = w.v0;
        const int32_t own_lo = int32_t(std::lower_bound(vm.begin(), vm.begin() + s.nv_nb, v0) - vm.begin());
        BlockHdr hdr{s.n_ext, s.n_own, s.n_halo, s.nv_loc, own_lo, s.nv_own, w.t_base, v0, s.nv_nb, s.n_bnd,
                     w.part, 0};
        memcpy(blk, &hdr, sizeof(hdr));
        memcpy(blk + kHdrWords, vm.data(), vm.size() * 4);
        int32_t *tmap = blk + blk_tmap_off(s.nv_loc);
        for (int64_t i = 0; i < w.n_ext; ++i) tmap[i] = w.ext[i];
        for (int64_t i = 0; i < w.n_halo; ++i) tmap[w.n_ext + i] = w.halo[i];
        if (w.part)
            for (int64_t i = 0; i < w.n_int; ++i) tmap[w.n_ext + w.n_halo + i] = w.itet(i);
        uint16_t *lrows = reinterpret_cast<uint16_t *>(blk + blk_rows_off(s.nv_loc, s.n_ext, s.n_halo, s.xmap));
        // local id = position in vm: a table of vm's values in order
        thread_local DistinctIds pos;
        pos.reset(vm.size());
        for (int32_t v : vm) pos.add(v);
        auto local = [&](int32_t v) -> uint16_t {
            if (v >= v0 && v < v0 + s.nv_own) return uint16_t(own_lo + (v - v0));
            return uint16_t(pos.index(v));
        };
        int64_t li = 0;
        auto put = [&](int32_t t) {
            const int32_t *r = rows + 4 * int64_t(t);
            for (int j = 0; j < 4; ++j) lrows[4 * li + j] = local(r[j]);
            ++li;
        };
        for (int64_t i = 0; i < w.n_ext; ++i) put(w.ext[i]);
        for (int64_t i = 0; i < w.n_int; ++i) put(w.itet(i));
        for (int64_t i = 0; i < w.n_halo; ++i) put(w.halo[i]);
        uint16_t *bnd =
            reinterpret_cast<uint16_t *>(blk + blk_bnd_off(s.nv_loc, s.n_ext, s.n_own, s.n_halo, s.xmap));
        int32_t nb = 0;
        const int32_t v1 = v0 + s.nv_own;
        for (int64_t i = 0; i < w.n_int; ++i) {
            const int32_t *r = rows + 4 * int64_t(w.itet(i));
            if (r[0] >= v0 && r[0] < v1 && r[1] >= v1) bnd[nb++] = uint16_t(i);
        }
    };
    auto cluster_set = [&](int32_t k) {
        WSet w;
        w.v0 = hm.I_V[k];
        w.v1 = hm.I_V[k + 1];
        w.ext = hm.ext.data() + hm.ext_off[k];
        w.n_ext = hm.ext_off[k + 1] - hm.ext_off[k];
        w.t0 = hm.I_T[k];
        w.t1 = hm.I_T[k + 1];
        w.n_int = w.t1 - w.t0;
        w.halo = hm.halo.data() + hm.halo_off[k];
        w.n_halo = hm.halo_off[k + 1] - hm.halo_off[k];
        w.t_base = hm.I_T[k];
        return w;
    };
    hm.stats.assign(K, ClusterStat{});
    std::vector<std::vector<int32_t>> vmaps(K);
    std::atomic<int64_t> bad_k{-1};
    std::atomic<int64_t> dup_k{-1};
    parallel_dynamic(K, P, 16, [&](int64_t k, int) {
        const int rc = ws_scan(cluster_set(int32_t(k)), hm.stats[k], vmaps[k]);
        if (rc == 1) bad_k = k;
        if (rc == 2) dup_k = k;
    });
    if (dup_k >= 0) {
        err = "two tets have the same vertex set (cluster " + std::to_string(dup_k.load()) + ")";
        return false;
    }
    if (bad_k >= 0) {
        err = "cluster " + std::to_string(bad_k.load()) +
              " has a working set larger than 65535 local vertices or 65534 tets; use smaller clusters";
        return false;
    }

    // Clusters whose working set would not fit one CTA's shared memory are
    // also cut into parts of about part_v own vertices (contiguous ranges);
    // batched builds run the parts, each on its own CTA, instead of the
    // cluster.  A cluster whose parts would still not fit is cut again into
    // twice as many.
    const int32_t part_v = d.part_vertices > 0 ? d.part_vertices : kPartVertices;
    const int64_t cut_bytes = d.cut_bytes > 0 ? d.cut_bytes : kCutBytes;
    std::vector<int32_t> cutk;
    for (int32_t k = 0; k < K; ++k) {
        const ClusterStat &s = hm.stats[k];
        if (d.part_vertices >= 0 && s.nv_own >= 2 && estimate_smem(s, 512) > cut_bytes) cutk.push_back(k);
    }
    struct PartBuild {
        int32_t a0 = 0, a1 = 0, n_rows = 0;
        std::vector<int32_t> ext, in, halo, vm;
        ClusterStat s{};
    };
    std::vector<std::vector<PartBuild>> built(cutk.size());
    std::atomic<int64_t> bad_p{-1};
    // part [a0, a1) of cluster k: its working set and block facts
    auto make_part = [&](int32_t k, int32_t a0, int32_t a1, int32_t part_tag, PartBuild &pb) -> bool {
        pb = PartBuild{};
        pb.a0 = a0;
        pb.a1 = a1;
        auto touches = [&](int32_t t) {
            const int32_t *r = rows + 4 * int64_t(t);
            return (r[0] >= a0 && r[0] < a1) || (r[1] >= a0 && r[1] < a1) || (r[2] >= a0 && r[2] < a1) ||
                   (r[3] >= a0 && r[3] < a1);
        };
        for (int64_t i = hm.ext_off[k]; i < hm.ext_off[k + 1]; ++i)
            if (touches(hm.ext[i])) pb.ext.push_back(hm.ext[i]);
        for (int32_t t = hm.I_T[k]; t < hm.I_T[k + 1]; ++t)
            if (touches(t)) {
                pb.in.push_back(t);
                const int32_t *r = rows + 4 * int64_t(t);
                pb.n_rows += (r[0] >= a0 && r[0] < a1);
            }
        if (want_tt) {
            // tets across the face (b, c, d) of a row's tet (a, b, c, d) when
            // that face has no vertex in the part and they have none either
            for (int32_t t : pb.in) {
                const int32_t *r = rows + 4 * int64_t(t);
                if (r[0] < a0 || r[0] >= a1 || r[1] < a1) continue;
                const int32_t b = r[1], c = r[2], dd = r[3];
                for (int64_t q = vs_off[b]; q < vs_off[b + 1]; ++q) {
                    const int32_t u = order[q];
                    if (u == t) continue;
                    const int32_t *ru = rows + 4 * int64_t(u);
                    bool hc = false, hd = false, inp = false;
                    for (int j = 0; j < 4; ++j) {
                        hc |= ru[j] == c;
                        hd |= ru[j] == dd;
                        inp |= ru[j] >= a0 && ru[j] < a1;
                    }
                    if (hc && hd && !inp) pb.halo.push_back(u);
                }
            }
            std::sort(pb.halo.begin(), pb.halo.end());
            pb.halo.erase(std::unique(pb.halo.begin(), pb.halo.end()), pb.halo.end());
        }
        WSet w;
        w.v0 = a0;
        w.v1 = a1;
        w.ext = pb.ext.data();
        w.n_ext = int64_t(pb.ext.size());
        w.ilist = pb.in.data();
        w.n_int = int64_t(pb.in.size());
        w.halo = pb.halo.data();
        w.n_halo = int64_t(pb.halo.size());
        w.part = part_tag;
        w.t_base = hm.I_T[k];
        return ws_scan(w, pb.s, pb.vm) == 0;
    };
    parallel_dynamic(int64_t(cutk.size()), P, 1, [&](int64_t i, int) {
        const int32_t k = cutk[i], v0 = hm.I_V[k], nvo = hm.stats[k].nv_own;
        int32_t S = std::max(2, (nvo + part_v - 1) / part_v);
        for (;;) {
            std::vector<PartBuild> &pbs = built[i];
            pbs.assign(size_t(S), PartBuild{});
            bool fit = true;
            for (int32_t j = 0; j < S; ++j) {
                const int32_t a0 = v0 + int32_t(int64_t(nvo) * j / S), a1 = v0 + int32_t(int64_t(nvo) * (j + 1) / S);
                if (!make_part(k, a0, a1, 1, pbs[j])) {
                    bad_p = k;
                    return;
                }
                fit &= estimate_smem(pbs[j].s, 512) <= kPartFitBytes;
            }
            if (fit || S >= nvo) break;
            S = std::min(nvo, 2 * S);
        }
    });
    if (bad_p >= 0) {
        err = "a part of cluster " + std::to_string(bad_p.load()) + " has too large a working set";
        return false;
    }
    // parts numbered cluster by cluster, in vertex order
    hm.part_first.assign(size_t(K) + 1, 0);
    int32_t NP = 0;
    {
        size_t c = 0;
        for (int32_t k = 0; k < K; ++k) {
            hm.part_first[k] = NP;
            if (c < cutk.size() && cutk[c] == k) NP += int32_t(built[c++].size());
        }
        hm.part_first[K] = NP;
    }
    hm.NP = NP;
    hm.parts.assign(size_t(NP), PartInfo{});
    hm.stats.resize(size_t(K) + NP);
    vmaps.resize(size_t(K) + NP);
    std::vector<std::vector<int32_t>> pext(NP), pint(NP), phalo(NP);
    std::vector<std::array<int32_t, 3>> pr(NP);  // (cluster, first own vertex, end)
    for (size_t c = 0; c < cutk.size(); ++c) {
        const int32_t k = cutk[c];
        for (size_t j = 0; j < built[c].size(); ++j) {
            PartBuild &pb = built[c][j];
            const int32_t p = hm.part_first[k] + int32_t(j);
            pr[p] = {k, pb.a0, pb.a1};
            pb.s.xmap = pb.s.n_own;
            hm.stats[size_t(K) + p] = pb.s;
            vmaps[size_t(K) + p].swap(pb.vm);
            pext[p].swap(pb.ext);
            pint[p].swap(pb.in);
            phalo[p].swap(pb.halo);
            PartInfo &pi = hm.parts[p];
            pi.k = k;
            pi.x0 = pb.a0 - hm.I_V[k];
            pi.nvo = pb.a1 - pb.a0;
            pi.last = j + 1 == built[c].size() ? 1 : 0;
            pi.n_rows = pb.n_rows;
            pi.n_own_c = hm.I_T[k + 1] - hm.I_T[k];
            pi.t_base_c = hm.I_T[k];
        }
    }
    std::vector<std::vector<PartBuild>>().swap(built);
    auto part_set = [&](int32_t p) {
        WSet w;
        w.v0 = pr[p][1];
        w.v1 = pr[p][2];
        w.ext = pext[p].data();
        w.n_ext = int64_t(pext[p].size());
        w.ilist = pint[p].data();
        w.n_int = int64_t(pint[p].size());
        w.halo = phalo[p].data();
        w.n_halo = int64_t(phalo[p].size());
        w.part = p + 1;
        w.t_base = hm.I_T[pr[p][0]];
        return w;
    };
    std::vector<int32_t>().swap(order);
    std::vector<int64_t>().swap(vs_off);

    const int64_t NI = int64_t(K) + NP;
    hm.blk_off.assign(size_t(NI) + 1, 0);
    int64_t run = 0;
    hm.ext_total = 0;
    hm.halo_total = 0;
    for (int64_t i = 0; i < NI; ++i) {
        const ClusterStat &s = hm.stats[i];
        hm.blk_off[i] = run;
        run += blk_words(s.nv_loc, s.n_ext, s.n_own, s.n_halo, s.n_bnd, s.xmap);
        if (i < K) {
            hm.ext_total += s.n_ext;
            hm.halo_total += s.n_halo;
        }
    }
    hm.blk_off[NI] = run;
    hm.blocks_words = run;
    if (!hm.alloc_blocks(run)) {
        err = "host allocation of the cluster blocks failed";
        return false;
    }
    parallel_dynamic(NI, P, 16, [&](int64_t i, int) {
        const WSet w = i < K ? cluster_set(int32_t(i)) : part_set(int32_t(i - K));
        ws_fill(w, hm.stats[i], vmaps[i], hm.blocks + hm.blk_off[i], hm.blk_off[i + 1] - hm.blk_off[i]);
    });
    hm.host_seconds = std::chrono::duration<double>(clk::now() - t0).count();
    return true;
}

}  // namespace gale
