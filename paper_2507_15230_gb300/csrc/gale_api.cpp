// C ABI: context life cycle, loading, bulk builds, views and exports.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <thread>

#include "gale_ctx.h"
#include "gale_par.h"

using gale::WorkItem;

namespace gale {

static thread_local std::string t_error;

void set_error(const std::string &msg) { t_error = msg; }

// Serving hooks (gale_serve.cpp).
void serve_destroy(gale_ctx *ctx);

}  // namespace gale

namespace {

constexpr int32_t kMaxExportChunks = 64;  // pipelined build + export

gale_status fail(gale_status s, const std::string &msg) {
    gale::set_error(msg);
    return s;
}

gale_status cuda_fail(cudaError_t e, const char *what) {
    return fail(GALE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(call)                                       \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);  \
    } while (0)

int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

gale::Caps merge(const gale::Caps &a, const gale::Caps &b) {
    gale::Caps c{};
    c.blk_words = std::max(a.blk_words, b.blk_words);
    c.nv_own = std::max(a.nv_own, b.nv_own);
    c.n_vt = std::max(a.n_vt, b.n_vt);
    c.n_own = std::max(a.n_own, b.n_own);
    c.nv_loc = std::max(a.nv_loc, b.nv_loc);
    c.nv_nb = std::max(a.nv_nb, b.nv_nb);
    c.max_deg = std::max(a.max_deg, b.max_deg);
    c.max_vv = std::max(a.max_vv, b.max_vv);
    c.max_e = std::max(a.max_e, b.max_e);
    c.max_etv = std::max(a.max_etv, b.max_etv);
    c.max_tt = std::max(a.max_tt, b.max_tt);
    c.max_up = std::max(a.max_up, b.max_up);
    c.hcap = std::max(a.hcap, b.hcap);
    c.n_tot = std::max(a.n_tot, b.n_tot);
    c.n_star = std::max(a.n_star, b.n_star);
    return c;
}

// Block size for a cluster: every phase spreads its work over all threads,
// so the size follows the cluster's tet count (about five tets per thread),
// a power of two in [64, 512] (a tuning override applies when set).
int threads_for(const gale_ctx *ctx, const gale::ClusterStat &s) {
    if (ctx->threads_override > 0) return ctx->threads_override;
    const int64_t want = (int64_t(s.n_ext) + s.n_own) / 5;
    int t = 64;
    while (t < 512 && t < want) t <<= 1;
    return t;
}

// Size bins: work items (clusters, then the parts of cut clusters) sorted by
// shared-memory need, cut where the merged plan would cross the next
// occupancy tier (4, 3, 2, 1 CTAs per SM).  Items whose plan exceeds the
// shared memory of one CTA go to spill bins: the same kernel with its
// regions in a per-CTA slice of global scratch.  Cut clusters get bins of
// their own, which batched builds skip (they run the parts).  Non-manifold
// clusters (the counting pass marks them) get per-item bins of their own:
// the hot shared-memory kernel leaves out the general TT pass they need.
gale_status plan_bins(gale_ctx *ctx, bool with_sizes) {
    const int32_t K = ctx->hm.K;
    const int32_t NI = K + ctx->hm.NP;
    // dynamic shared memory a CTA may plan for: the opt-in limit less the
    // kernels' static shared memory
    constexpr int kStaticMargin = 512;
    const int smem_cta = gale::dynamic_smem_limit();
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device);
    auto caps_k = [&](int32_t k) {
        return gale::caps_of(ctx->hm.stats[k], with_sizes ? ctx->sizes.data() + size_t(5) * k : nullptr);
    };
    std::vector<int32_t> need(NI), thr(NI);
    std::vector<uint8_t> big(NI), cut(NI, 0), gen(NI, 0);
    for (int32_t k = 0; k < NI; ++k) {
        if (ctx->hm.stats[k].max_up > 255)
            return fail(GALE_EINVAL, "cluster " + std::to_string(k < K ? k : ctx->hm.parts[k - K].k) +
                                         " has a vertex with more than 255 upper neighbours (unsupported)");
        thr[k] = threads_for(ctx, ctx->hm.stats[k]);
        need[k] = gale::plan_smem(caps_k(k), thr[k]).total;
        big[k] = need[k] > smem_cta;
        if (k < K) cut[k] = ctx->hm.part_first[k + 1] > ctx->hm.part_first[k];
        if (with_sizes && k < K && size_t(k) < ctx->tt_general.size()) gen[k] = ctx->tt_general[k] != 0 && !big[k];
    }
    std::vector<int32_t> idx(NI);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
        if (cut[a] != cut[b]) return cut[a] < cut[b];
        if (big[a] != big[b]) return big[a] < big[b];
        if (gen[a] != gen[b]) return gen[a] < gen[b];
        return thr[a] != thr[b] ? thr[a] < thr[b] : need[a] < need[b];
    });
    std::vector<int> tiers;
    for (int per = 4; per >= 1; --per) tiers.push_back(std::min(smem_sm / per - 1024 - kStaticMargin, smem_cta));
    ctx->bins.clear();
    ctx->bin_of.assign(NI, -1);
    size_t tier = 0;
    int cur_thr = 0;
    bool cur_big = false, cur_cut = false, cur_gen = false;
    gale::Caps cur{};
    std::vector<int32_t> members;
    auto close = [&]() {
        if (members.empty()) return;
        gale::Bin b;
        b.plan = gale::plan_smem(cur, cur_thr);
        b.spill = cur_big;
        b.cut = cur_cut;
        b.tt_general = cur_gen;
        std::stable_sort(members.begin(), members.end(),
                         [&](int32_t a, int32_t c) { return need[a] > need[c]; });  // largest first
        b.clusters = members;
        for (int32_t k : members) ctx->bin_of[k] = int32_t(ctx->bins.size());
        ctx->bins.push_back(std::move(b));
        members.clear();
        cur = gale::Caps{};
    };
    for (int32_t k : idx) {
        if (!members.empty() && (thr[k] != cur_thr || bool(big[k]) != cur_big || bool(cut[k]) != cur_cut ||
                                 bool(gen[k]) != cur_gen)) {
            close();
            tier = 0;
        }
        cur_thr = thr[k];
        cur_big = big[k];
        cur_cut = cut[k];
        cur_gen = gen[k];
        gale::Caps m = members.empty() ? caps_k(k) : merge(cur, caps_k(k));
        if (!cur_big) {
            int tot = gale::plan_smem(m, cur_thr).total;
            while (tier < tiers.size() && tot > tiers[tier]) {
                close();
                ++tier;
                m = caps_k(k);
                tot = gale::plan_smem(m, cur_thr).total;
            }
            if (tier >= tiers.size()) tier = tiers.size() - 1;
        } else if (!members.empty() && gale::plan_smem(m, cur_thr).total > 2 * need[k]) {
            // spill bins: keep the merged plan within twice a member's own
            close();
            m = caps_k(k);
        }
        cur = m;
        members.push_back(k);
    }
    close();
    // The bins of the one-CTA-per-SM tier hold the largest clusters: merged
    // caps (each field's maximum over the members) soon exceed a CTA's shared
    // memory, which leaves many bins of a few clusters each, launched one
    // after another.  They become one bin per block size whose members each
    // keep their own plan (one persistent launch, the largest member's
    // shared memory).
    ctx->h_plans.assign(size_t(NI), gale::SmemPlan{});
    {
        // (block size, bin of cut clusters) -> bins of the top tier
        using Key = std::pair<int, bool>;
        std::map<Key, int> ntop;
        for (auto &b : ctx->bins)
            if (!b.spill && !b.tt_general && b.plan.total > tiers[2]) ntop[Key(b.plan.threads, b.cut)]++;
        std::vector<gale::Bin> kept;
        std::map<Key, gale::Bin> top;  // merged bins
        for (auto &b : ctx->bins) {
            if (b.tt_general) {  // each member under its own plan, in build_kernel_pi
                for (int32_t k : b.clusters) ctx->h_plans[k] = gale::plan_smem(caps_k(k), b.plan.threads);
                b.per_item = true;
                kept.push_back(std::move(b));
                continue;
            }
            if (b.spill || b.plan.total <= tiers[2] || ntop[Key(b.plan.threads, b.cut)] < 2) {
                kept.push_back(std::move(b));
                continue;
            }
            gale::Bin &t = top[Key(b.plan.threads, b.cut)];
            t.cut = b.cut;
            const bool first = t.clusters.empty();
            for (int32_t k : b.clusters) {
                ctx->h_plans[k] = gale::plan_smem(caps_k(k), b.plan.threads);
                if (first && t.clusters.empty()) t.plan = ctx->h_plans[k];
                else t.plan.caps = merge(t.plan.caps, ctx->h_plans[k].caps);
                t.plan.total = std::max(t.plan.total, ctx->h_plans[k].total);
                t.clusters.push_back(k);
            }
            t.per_item = true;
        }
        for (auto &kv : top) {
            gale::Bin &t = kv.second;
            std::stable_sort(t.clusters.begin(), t.clusters.end(),
                             [&](int32_t a, int32_t c) { return need[a] > need[c]; });  // largest first
            kept.push_back(std::move(t));
        }
        ctx->bins = std::move(kept);
        for (size_t b = 0; b < ctx->bins.size(); ++b)
            for (int32_t k : ctx->bins[b].clusters) ctx->bin_of[k] = int32_t(b);
    }
    if (!ctx->d_plans) {
        ctx->d_plans = static_cast<gale::SmemPlan *>(ctx->dalloc(sizeof(gale::SmemPlan) * size_t(std::max(NI, 1))));
        if (!ctx->d_plans) return fail(GALE_ENOMEM, "device allocation of the per-cluster plans failed");
    }
    if (NI > 0 &&
        cudaMemcpy(ctx->d_plans, ctx->h_plans.data(), sizeof(gale::SmemPlan) * size_t(NI), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return fail(GALE_ECUDA, "uploading the per-cluster plans failed");
    if (int(ctx->bins.size()) > gale::kMaxBins)
        return fail(GALE_EINVAL, "the working sets fall into more than " + std::to_string(gale::kMaxBins) +
                                     " size bins; use more even clusters");
    int max_total = 0;
    for (auto &b : ctx->bins)
        if (!b.spill) max_total = std::max(max_total, b.plan.total);
    if (!gale::prepare_kernels(max_total))
        return fail(GALE_ECUDA, "setting the kernels' shared memory limit failed");
    int64_t spill_need = 0;
    for (auto &b : ctx->bins) {
        int per_sm = gale::max_ctas_per_sm(b.plan, b.spill, b.per_item);
        if (per_sm < 1 && !b.spill && !b.per_item) {
            b.spill = true;  // cannot launch with this much shared memory: run in global scratch
            per_sm = gale::max_ctas_per_sm(b.plan, true);
        }
        if (per_sm < 1) return fail(GALE_EINVAL, "a size bin cannot be launched (threads or registers)");
        if (ctx->ctas_override > 0) per_sm = std::min(per_sm, ctx->ctas_override);
        if (b.spill) per_sm = std::min(per_sm, 2);  // bounds the scratch footprint
        b.ctas_per_sm = per_sm;
        b.grid = std::max(1, std::min<int>(int(b.clusters.size()), per_sm * ctx->sm_count));
        if (b.spill) spill_need = std::max<int64_t>(spill_need, int64_t(b.grid) * b.plan.total);
    }
    if (spill_need > ctx->spill_bytes) {
        if (ctx->d_spill) ctx->dfree(ctx->d_spill);
        ctx->d_spill = static_cast<char *>(ctx->dalloc(size_t(spill_need)));
        ctx->spill_bytes = ctx->d_spill ? spill_need : 0;
        if (!ctx->d_spill) return fail(GALE_ENOMEM, "device allocation of the large-cluster scratch failed");
    }
    return GALE_OK;
}

char *scratch_of(gale_ctx *ctx, const gale::Bin &b) { return b.spill ? ctx->d_spill : nullptr; }
// build capacities of cluster k (its exact sizes known)
gale::Caps bin_caps(const gale_ctx *ctx, int32_t k) {
    return gale::caps_of(ctx->hm.stats[k], ctx->sizes.data() + size_t(5) * k);
}
const gale::SmemPlan *plans_of(gale_ctx *ctx, const gale::Bin &b) { return b.per_item ? ctx->d_plans : nullptr; }
// persistent grid of a launch over n members (a team launch holds `teams` of them per CTA)
int grid_of(const gale::Bin &b, int32_t n) {
    const int32_t need = b.teams > 0 ? (n + b.teams - 1) / b.teams : n;
    return std::max(1, std::min<int>(b.grid, need));
}
// bins whose batched launches may run several clusters per CTA: small
// whole clusters under one merged plan in shared memory
bool team_eligible(const gale_ctx *ctx, const gale::Bin &b) {
    if (b.spill || b.per_item || b.cut) return false;
    for (int32_t k : b.clusters)
        if (k >= ctx->hm.K) return false;
    return true;
}

}  // namespace

namespace gale {
// Plans of the serving loop.  The loop's CTAs build any cluster under the
// cluster's own plan at one block size (the largest of the size bins), so
// every bin whose members each fit one CTA is served by the loop; the others
// (global-scratch bins) are served by batched launches beside it.  Returns
// the launch envelope (block size, the largest member's shared memory);
// *fits = some bin made it; (*in_loop)[b] marks the bins the loop serves;
// own (optional, K entries) receives the plans of their members.
SmemPlan serve_plan(gale_ctx *ctx, bool *fits, std::vector<uint8_t> *in_loop, std::vector<SmemPlan> *own) {
    const size_t nb = ctx->bins.size();
    const int32_t K = ctx->hm.K;
    const int limit = dynamic_smem_limit();
    int threads = 64;
    for (size_t b = 0; b < nb; ++b)
        if (!ctx->bins[b].spill) threads = std::max(threads, ctx->bins[b].plan.threads);
    std::vector<uint8_t> sel(nb, 0);
    if (own) own->assign(size_t(K), SmemPlan{});
    SmemPlan env = plan_smem(Caps{}, threads);
    env.total = 0;
    bool any = false;
    for (size_t b = 0; b < nb; ++b) {
        const Bin &bin = ctx->bins[b];
        if (bin.spill) continue;
        int top = 0;
        for (int32_t k : bin.clusters)
            if (k < K) top = std::max(top, plan_smem(bin_caps(ctx, k), threads).total);
        if (top > limit) continue;
        SmemPlan probe = env;
        probe.total = std::max(env.total, top);
        if (serve_ctas_per_sm(probe) < 1) continue;
        env.total = probe.total;
        sel[b] = 1;
        any = true;
        if (own)
            for (int32_t k : bin.clusters)
                if (k < K) (*own)[k] = plan_smem(bin_caps(ctx, k), threads);
    }
    *fits = any;
    if (in_loop) *in_loop = sel;
    return env;
}
// Lengths of the ten output arrays of cluster k under mask.
void item_lengths(const gale_ctx *ctx, int32_t k, uint32_t mask, int64_t *L) {
    const int64_t *sz = ctx->sizes.data() + size_t(5) * k;
    const int64_t nvo = ctx->hm.I_V[k + 1] - ctx->hm.I_V[k];
    const int64_t nown = ctx->hm.I_T[k + 1] - ctx->hm.I_T[k];
    const bool vt = mask & GALE_VT, vv = mask & GALE_VV, et = mask & GALE_ET, tt = mask & GALE_TT;
    L[0] = vt ? nvo + 1 : 0;
    L[1] = vt ? sz[0] : 0;
    L[2] = vv ? nvo + 1 : 0;
    L[3] = vv ? sz[1] : 0;
    L[4] = et ? nvo + 1 : 0;
    L[5] = et ? sz[2] : 0;
    L[6] = et ? sz[2] + 1 : 0;
    L[7] = et ? sz[3] : 0;
    L[8] = tt ? nown + 1 : 0;
    L[9] = tt ? sz[4] : 0;
}
}  // namespace gale

namespace {

// Per bin, its members' item ids (the counting pass) and their positions in
// the full build's item list (batched full builds; -1 for cut clusters,
// whose bins those builds skip).
gale_status upload_orders(gale_ctx *ctx) {
    std::vector<int32_t> ids, pos;
    ctx->order_all_off.assign(1, 0);
    for (auto &b : ctx->bins) {
        for (int32_t k : b.clusters) {
            ids.push_back(k);
            pos.push_back(ctx->pos_all[k]);
        }
        ctx->order_all_off.push_back(int64_t(ids.size()));
    }
    CUDA_TRY(cudaMemcpyAsync(ctx->d_order_ids, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(ctx->d_order_all, pos.data(), pos.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));  // the host vectors go out of scope
    return GALE_OK;
}

gale::DevMesh dev_mesh(gale_ctx *ctx) {
    gale::DevMesh m{ctx->d_blocks, ctx->d_blk_off, ctx->d_I_V, ctx->d_I_T, ctx->hm.K};
    m.NP = ctx->hm.NP;
    m.parts = ctx->d_parts;
    m.tt_pos = ctx->d_tt_pos;
    m.tt_general = ctx->d_tt_general;
    return m;
}

// The item list of a batched build of the listed clusters: every cut
// cluster replaced by its parts, in order.
std::vector<int32_t> expand_items(const gale_ctx *ctx, const std::vector<int32_t> &list) {
    if (ctx->hm.NP == 0) return list;
    std::vector<int32_t> out;
    out.reserve(list.size());
    const int32_t K = ctx->hm.K;
    for (int32_t k : list) {
        const int32_t p0 = ctx->hm.part_first[k], p1 = ctx->hm.part_first[k + 1];
        if (p1 == p0) out.push_back(k);
        for (int32_t p = p0; p < p1; ++p) out.push_back(K + p);
    }
    return out;
}

gale_status check_device_error(gale_ctx *ctx) {
    int32_t e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, ctx->d_err, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    ctx->last_err_word = e;
    if (e == 0) return GALE_OK;
    CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, 4, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    std::string msg = "kernel error word " + std::to_string(e) + ":";
    if (e & gale::ERR_CAPACITY) msg += " cluster exceeded its launch capacities;";
    if (e & gale::ERR_NONMANIFOLD) msg += " a triangle of a cluster cut into parts lies in more than two tets (parts need a manifold mesh);";
    if (e & gale::ERR_HASH_FULL) msg += " face hash overflow;";
    if (e & gale::ERR_BAD_ITEM) msg += " bad cluster id in a work item;";
    if (e & gale::ERR_TIMEOUT) msg += " a device wait timed out;";
    return fail(GALE_EDEVICE, msg);
}

gale_status count_pass(gale_ctx *ctx) {
    const int32_t K = ctx->hm.K, NP = ctx->hm.NP, NI = K + NP;
    CUDA_TRY(cudaMemsetAsync(ctx->d_sizes, 0, sizeof(int64_t) * 5 * NI, ctx->stream));
    CUDA_TRY(cudaMemsetAsync(ctx->d_tt_general, 0, sizeof(int32_t) * std::max(K, 1), ctx->stream));
    for (size_t b = 0; b < ctx->bins.size(); ++b) {
        const gale::Bin &bin = ctx->bins[b];
        int rc = gale::launch_count_pass(dev_mesh(ctx), bin.plan, ctx->d_order_ids + ctx->order_all_off[b],
                                         int32_t(bin.clusters.size()), ctx->d_sizes, ctx->d_err,
                                         ctx->d_tickets + b, bin.grid, ctx->stream, scratch_of(ctx, bin),
                                         ctx->precond, plans_of(ctx, bin));
        if (rc != 0) return cuda_fail(cudaError_t(rc), "count pass launch");
    }
    gale_status st = check_device_error(ctx);
    if (st != GALE_OK) return st;
    ctx->sizes.resize(size_t(5) * NI);
    CUDA_TRY(cudaMemcpyAsync(ctx->sizes.data(), ctx->d_sizes, sizeof(int64_t) * 5 * NI, cudaMemcpyDeviceToHost,
                             ctx->stream));
    ctx->tt_general.assign(size_t(K), 0);
    if (K > 0)
        CUDA_TRY(cudaMemcpyAsync(ctx->tt_general.data(), ctx->d_tt_general, sizeof(int32_t) * K,
                                 cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (int a = 0; a < 5; ++a) ctx->totals[a] = 0;
    for (int32_t k = 0; k < K; ++k)
        for (int a = 0; a < 5; ++a) ctx->totals[a] += ctx->sizes[size_t(5) * k + a];
    if (NP == 0) return GALE_OK;
    // Parts: the cluster-level values at each part's start, checked against
    // the cluster's own count; the TT row offsets of every internal tet of a
    // cut cluster from the row lengths the parts counted.
    auto &hm = ctx->hm;
    const bool tt = (ctx->precond & GALE_TT) != 0;
    std::vector<int32_t> len;
    if (tt) {
        len.resize(size_t(hm.nt));
        CUDA_TRY(cudaMemcpy(len.data(), ctx->d_tt_pos, sizeof(int32_t) * size_t(hm.nt), cudaMemcpyDeviceToHost));
    }
    for (int32_t k = 0; k < K; ++k) {
        const int32_t p0 = hm.part_first[k], p1 = hm.part_first[k + 1];
        if (p1 == p0) continue;
        int64_t run[5] = {}, rows = 0;
        for (int32_t p = p0; p < p1; ++p) {
            gale::PartInfo &pi = hm.parts[p];
            const int64_t *sz = ctx->sizes.data() + size_t(5) * (K + p);
            pi.b_vt = int32_t(run[0]);
            pi.b_vv = int32_t(run[1]);
            pi.b_e = int32_t(run[2]);
            pi.b_et = int32_t(run[3]);
            pi.b_tt = int32_t(run[4]);
            pi.b_to = int32_t(rows);
            for (int a = 0; a < 5; ++a) run[a] += sz[a];
            rows += pi.n_rows;
            pi.tt_total = int32_t(ctx->sizes[size_t(5) * k + 4]);
        }
        for (int a = 0; a < 5; ++a)
            if (run[a] != ctx->sizes[size_t(5) * k + a] && (a < 4 || tt))
                return fail(GALE_EDEVICE, "the parts of cluster " + std::to_string(k) +
                                              " disagree with the cluster's own sizes");
        if (rows != hm.I_T[k + 1] - hm.I_T[k])
            return fail(GALE_EDEVICE, "the parts of cluster " + std::to_string(k) + " miss internal tets");
        if (tt) {
            int64_t pos = 0;
            for (int32_t t = hm.I_T[k]; t < hm.I_T[k + 1]; ++t) {
                const int32_t l = len[t];
                if (l < 0 || l > 4) return fail(GALE_EDEVICE, "a part reported a bad TT row length");
                len[t] = int32_t(pos);
                pos += l;
            }
            if (pos != ctx->sizes[size_t(5) * k + 4])
                return fail(GALE_EDEVICE, "the parts of cluster " + std::to_string(k) + " disagree on TT");
        }
    }
    if (tt)
        CUDA_TRY(cudaMemcpy(ctx->d_tt_pos, len.data(), sizeof(int32_t) * size_t(hm.nt), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(ctx->d_parts, hm.parts.data(), sizeof(gale::PartInfo) * size_t(NP), cudaMemcpyHostToDevice));
    return GALE_OK;
}


// Launch order of listed items (clusters, and the parts that stand for cut
// clusters), chunk by chunk and, within a chunk, bin by bin, each bin's
// members in the bin's largest-first order: the positions of chunk c's
// members relative to cut[c], in order[boff[c][b] .. boff[c][b+1]).  Bins of
// cut clusters get no entries.  One pass over the bins' member lists, no
// sorting (list positions are pos_of[k], or pos_all[k] when the list is the
// full build's).  False if some listed item is in no bin.
bool chunk_bin_orders(const gale_ctx *ctx, const std::vector<int32_t> &list, bool all,
                      const std::vector<int32_t> &cut, std::vector<int32_t> &order,
                      std::vector<std::vector<int64_t>> &boff) {
    const int32_t NI = ctx->hm.K + ctx->hm.NP, cnt = int32_t(list.size());
    const int32_t chunks = int32_t(cut.size()) - 1;
    const size_t nb = ctx->bins.size();
    std::vector<int32_t> own_pos;
    if (!all) {
        own_pos.assign(NI, -1);
        for (int32_t i = 0; i < cnt; ++i) own_pos[list[i]] = i;
    }
    const std::vector<int32_t> &pos_of = all ? ctx->pos_all : own_pos;
    std::vector<int32_t> chunk_of(cnt);
    for (int32_t c = 0; c < chunks; ++c)
        for (int32_t i = cut[c]; i < cut[c + 1]; ++i) chunk_of[i] = c;
    std::vector<int64_t> count(size_t(chunks) * nb, 0);
    for (size_t b = 0; b < nb; ++b) {
        if (ctx->bins[b].cut) continue;
        for (int32_t k : ctx->bins[b].clusters) {
            const int32_t p = pos_of[k];
            if (p >= 0 && p < cnt) count[size_t(chunk_of[p]) * nb + b]++;
        }
    }
    boff.assign(chunks, std::vector<int64_t>(nb + 1, 0));
    std::vector<int64_t> fill(size_t(chunks) * nb);
    int64_t run = 0;
    for (int32_t c = 0; c < chunks; ++c) {
        for (size_t b = 0; b < nb; ++b) {
            boff[c][b] = run;
            fill[size_t(c) * nb + b] = run;
            run += count[size_t(c) * nb + b];
        }
        boff[c][nb] = run;
    }
    order.assign(size_t(run), 0);
    for (size_t b = 0; b < nb; ++b) {
        if (ctx->bins[b].cut) continue;
        for (int32_t k : ctx->bins[b].clusters) {
            const int32_t p = pos_of[k];
            if (p < 0 || p >= cnt) continue;
            const int32_t c = chunk_of[p];
            order[size_t(fill[size_t(c) * nb + b]++)] = p - cut[c];
        }
    }
    return run == cnt;
}

gale_status ensure_bulk(gale_ctx *ctx, const int64_t *need) {
    bool realloc = false;
    for (int a = 0; a < 10; ++a) {
        if (need[a] <= ctx->bulk_cap[a]) continue;
        if (ctx->bulk[a]) ctx->dfree(ctx->bulk[a]);
        ctx->bulk[a] = nullptr;
        ctx->bulk_cap[a] = 0;
        const int64_t cap = need[a] + need[a] / 16 + 64;
        ctx->bulk[a] = static_cast<int32_t *>(ctx->dalloc(size_t(cap) * 4));
        if (!ctx->bulk[a]) return fail(GALE_ENOMEM, "device allocation of a bulk output array failed");
        ctx->bulk_cap[a] = cap;
        realloc = true;
    }
    if (realloc) {
        for (auto &g : ctx->graphs)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
    // base pointers for every mask (unmasked arrays NULL)
    WorkItem base[16];
    for (uint32_t m = 0; m < 16; ++m) {
        WorkItem &w = base[m];
        memset(&w, 0, sizeof(w));
        w.vt_off = (m & GALE_VT) ? ctx->bulk[0] : nullptr;
        w.vt_val = (m & GALE_VT) ? ctx->bulk[1] : nullptr;
        w.vv_off = (m & GALE_VV) ? ctx->bulk[2] : nullptr;
        w.vv_val = (m & GALE_VV) ? ctx->bulk[3] : nullptr;
        w.eu_off = (m & GALE_ET) ? ctx->bulk[4] : nullptr;
        w.e_w = (m & GALE_ET) ? ctx->bulk[5] : nullptr;
        w.et_off = (m & GALE_ET) ? ctx->bulk[6] : nullptr;
        w.et_val = (m & GALE_ET) ? ctx->bulk[7] : nullptr;
        w.tt_off = (m & GALE_TT) ? ctx->bulk[8] : nullptr;
        w.tt_val = (m & GALE_TT) ? ctx->bulk[9] : nullptr;
    }
    CUDA_TRY(cudaMemcpyAsync(ctx->d_arrays_base, base, sizeof(base), cudaMemcpyHostToDevice, ctx->stream));
    return GALE_OK;
}

}  // namespace

void *gale_ctx::dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (alloc_fn) {
        p = alloc_fn(alloc_ctx, bytes);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) allocs.push_back(gale::DevAlloc{p, bytes});
    return p;
}

void gale_ctx::dfree(void *p) {
    if (!p) return;
    for (size_t i = 0; i < allocs.size(); ++i)
        if (allocs[i].ptr == p) {
            allocs.erase(allocs.begin() + i);
            break;
        }
    if (free_fn) free_fn(alloc_ctx, p);
    else cudaFree(p);
}

bool gale::HostMesh::alloc_blocks(int64_t words) {
    free_blocks();
    const size_t bytes = size_t(std::max<int64_t>(words, 4)) * 4;
    if (cudaHostAlloc(reinterpret_cast<void **>(&blocks), bytes, cudaHostAllocDefault) == cudaSuccess) {
        blocks_pinned = true;
        return true;
    }
    cudaGetLastError();
    blocks = static_cast<int32_t *>(malloc(bytes));
    blocks_pinned = false;
    return blocks != nullptr;
}

void gale::HostMesh::free_blocks() {
    if (!blocks) return;
    if (blocks_pinned) cudaFreeHost(blocks);
    else free(blocks);
    blocks = nullptr;
}

namespace gale {

namespace {
constexpr size_t kStageBytes = size_t(128) << 20;  // each of the two staging buffers
constexpr size_t kDirectBytes = size_t(32) << 20;  // below this a pageable copy goes straight through
}  // namespace

// Pageable destinations: the copy engine fills one staging buffer while the
// host threads move the other into place, each thread a fixed slice of every
// chunk (so the threads also share the first touch of the destination pages).
gale_status copy_to_host(gale_ctx *ctx, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return GALE_OK;
    cudaStream_t s = ctx->stream;
    cudaPointerAttributes at{};
    const bool locked = cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeHost;
    cudaGetLastError();  // an unregistered pointer may leave an error behind
    if (locked || bytes < kDirectBytes) {
        if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(GALE_ECUDA, "device to host copy failed");
        return GALE_OK;
    }
    std::lock_guard<std::mutex> lock(ctx->stage_mu);
    for (int b = 0; b < 2; ++b) {
        if (!ctx->stage[b] && cudaHostAlloc(&ctx->stage[b], kStageBytes, cudaHostAllocDefault) != cudaSuccess) {
            ctx->stage[b] = nullptr;
            cudaGetLastError();
            return fail(GALE_ENOMEM, "pinned staging allocation failed");
        }
        if (!ctx->stage_ev[b] && cudaEventCreateWithFlags(&ctx->stage_ev[b], cudaEventDisableTiming) != cudaSuccess) {
            ctx->stage_ev[b] = nullptr;
            return fail(GALE_ECUDA, "staging event creation failed");
        }
    }
    const int64_t nch = int64_t((bytes + kStageBytes - 1) / kStageBytes);
    const int T = std::max(1, std::min(host_threads(0), 32));
    auto chunk_len = [&](int64_t c) { return std::min(kStageBytes, bytes - size_t(c) * kStageBytes); };
    auto issue = [&](int64_t c) {
        return cudaMemcpyAsync(ctx->stage[c & 1], static_cast<const char *>(src) + size_t(c) * kStageBytes,
                               chunk_len(c), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
               cudaEventRecord(ctx->stage_ev[c & 1], s) == cudaSuccess;
    };
    std::atomic<int64_t> ready{-1};  // last chunk whose staging copy is complete
    std::atomic<int64_t> moved{0};   // slices moved into dst
    std::atomic<bool> stop{false};
    auto worker = [&](int t) {
        for (int64_t c = 0; c < nch; ++c) {
            while (ready.load(std::memory_order_acquire) < c) {
                if (stop.load(std::memory_order_acquire)) return;
                std::this_thread::yield();
            }
            const size_t len = chunk_len(c), lo = len * size_t(t) / size_t(T), hi = len * size_t(t + 1) / size_t(T);
            std::memcpy(static_cast<char *>(dst) + size_t(c) * kStageBytes + lo,
                        static_cast<const char *>(ctx->stage[c & 1]) + lo, hi - lo);
            moved.fetch_add(1, std::memory_order_acq_rel);
        }
    };
    bool ok = issue(0) && (nch < 2 || issue(1));
    std::vector<std::thread> th;
    try {
        th.reserve(size_t(T));
        for (int t = 0; t < T; ++t) th.emplace_back(worker, t);
    } catch (const std::exception &) {  // no threads to be had: copy straight through
        stop.store(true, std::memory_order_release);
        for (auto &x : th) x.join();
        cudaStreamSynchronize(s);
        if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(GALE_ECUDA, "device to host copy failed");
        return GALE_OK;
    }
    for (int64_t c = 0; ok && c < nch; ++c) {
        if (cudaEventSynchronize(ctx->stage_ev[c & 1]) != cudaSuccess) {
            ok = false;
            break;
        }
        ready.store(c, std::memory_order_release);
        // the buffer of chunk c takes chunk c + 2 once every thread moved its slice
        while (moved.load(std::memory_order_acquire) < int64_t(T) * (c + 1)) std::this_thread::yield();
        if (c + 2 < nch) ok = issue(c + 2);
    }
    if (!ok) stop.store(true, std::memory_order_release);
    for (auto &x : th) x.join();
    if (!ok) {
        cudaStreamSynchronize(s);
        return fail(GALE_ECUDA, "staged device to host copy failed");
    }
    return GALE_OK;
}

}  // namespace gale

extern "C" {

const char *gale_last_error(void) { return gale::t_error.c_str(); }

void gale_destroy(gale_ctx *ctx) {
    if (!ctx) return;
    gale::serve_destroy(ctx);
    gale::enumeration_destroy(ctx);
    gale::cobound_destroy(ctx);
    if (ctx->device >= 0) {
        cudaSetDevice(ctx->device);
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        for (auto &g : ctx->graphs)
            if (g) cudaGraphExecDestroy(g);
        if (ctx->copy_stream) {
            cudaStreamSynchronize(ctx->copy_stream);
            cudaStreamDestroy(ctx->copy_stream);
        }
        for (cudaEvent_t e : ctx->chunk_events) cudaEventDestroy(e);
        for (int b = 0; b < 2; ++b) {
            if (ctx->stage[b]) cudaFreeHost(ctx->stage[b]);
            if (ctx->stage_ev[b]) cudaEventDestroy(ctx->stage_ev[b]);
        }
        while (!ctx->allocs.empty()) ctx->dfree(ctx->allocs.back().ptr);
        if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
}

gale_status gale_load_mesh(const gale_mesh_desc *desc, gale_ctx **out) {
    if (!desc || !out) return fail(GALE_EINVAL, "NULL argument");
    *out = nullptr;
    if (desc->precondition_mask == 0 || (desc->precondition_mask & ~uint32_t(GALE_ALL)))
        return fail(GALE_EINVAL, "precondition_mask must be a non-empty subset of GALE_ALL");
    auto ctx = std::make_unique<gale_ctx>();
    ctx->precond = desc->precondition_mask;
    ctx->device = desc->device;
    ctx->alloc_fn = desc->alloc;
    ctx->free_fn = desc->free;
    ctx->alloc_ctx = desc->alloc_ctx;
    ctx->cache_budget = desc->cache_budget_bytes;
    std::string err;
    try {
        if (!gale::prepare_host(*desc, ctx->hm, err)) return fail(GALE_EINVAL, err);
    } catch (const std::bad_alloc &) {
        return fail(GALE_ENOMEM, "host allocation failed during initialisation");
    }
    if (ctx->device < 0) {
        *out = ctx.release();
        return GALE_OK;
    }
    auto t0 = std::chrono::steady_clock::now();
    CUDA_TRY(cudaSetDevice(ctx->device));
    if (desc->stream) {
        ctx->stream = static_cast<cudaStream_t>(desc->stream);
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    ctx->sm_count = gale::device_sm_count();
    const int32_t K = ctx->hm.K;
    auto &hm = ctx->hm;
    const int32_t NP = hm.NP, NI = K + NP;  // work items: clusters, then parts
    // the full build's item list: cut clusters replaced by their parts
    {
        std::vector<int32_t> all(K);
        std::iota(all.begin(), all.end(), 0);
        ctx->all_items = expand_items(ctx.get(), all);
        ctx->pos_all.assign(NI, -1);
        for (size_t i = 0; i < ctx->all_items.size(); ++i) ctx->pos_all[ctx->all_items[i]] = int32_t(i);
    }
    ctx->d_blocks = static_cast<int32_t *>(ctx->dalloc(size_t(hm.blocks_words) * 4));
    ctx->d_blk_off = static_cast<int64_t *>(ctx->dalloc(sizeof(int64_t) * (NI + 1)));
    ctx->d_I_V = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * (K + 1)));
    ctx->d_I_T = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * (K + 1)));
    ctx->d_sizes = static_cast<int64_t *>(ctx->dalloc(sizeof(int64_t) * 5 * NI));
    ctx->d_tt_general = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * std::max(K, 1)));
    ctx->d_err = static_cast<int32_t *>(ctx->dalloc(64));
    ctx->d_tickets = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * gale::kMaxBins));
    ctx->d_ids = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * NI));
    ctx->d_order_all = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * NI));
    ctx->d_order_ids = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * NI));
    ctx->d_order_part = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * NI));
    ctx->d_items = static_cast<WorkItem *>(ctx->dalloc(sizeof(WorkItem) * NI));
    ctx->d_arrays_base = static_cast<WorkItem *>(ctx->dalloc(sizeof(WorkItem) * 16));
    ctx->d_totals = static_cast<int64_t *>(ctx->dalloc(sizeof(int64_t) * 16));
    ctx->d_bsum = static_cast<int64_t *>(ctx->dalloc(sizeof(int64_t) * (gale::bases_scratch_words(NI) + 16)));
    if (NP > 0) {
        ctx->d_parts = static_cast<gale::PartInfo *>(ctx->dalloc(sizeof(gale::PartInfo) * NP));
        ctx->d_tt_pos = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * std::max<int64_t>(1, hm.nt)));
        ctx->d_all_items = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * ctx->all_items.size()));
    }
    if (!ctx->d_blocks || !ctx->d_blk_off || !ctx->d_I_V || !ctx->d_I_T || !ctx->d_sizes || !ctx->d_tt_general ||
        !ctx->d_err ||
        !ctx->d_tickets || !ctx->d_ids || !ctx->d_order_all || !ctx->d_order_ids || !ctx->d_order_part ||
        !ctx->d_items || !ctx->d_arrays_base || !ctx->d_totals || !ctx->d_bsum ||
        (NP > 0 && (!ctx->d_parts || !ctx->d_tt_pos || !ctx->d_all_items))) {
        gale_destroy(ctx.release());
        return fail(GALE_ENOMEM, "device allocation failed while loading the mesh");
    }
    CUDA_TRY(cudaMemcpyAsync(ctx->d_blocks, hm.blocks, size_t(hm.blocks_words) * 4, cudaMemcpyHostToDevice,
                             ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(ctx->d_blk_off, hm.blk_off.data(), sizeof(int64_t) * (NI + 1), cudaMemcpyHostToDevice,
                             ctx->stream));
    if (NP > 0) {
        // part records without the counted offsets (the counting pass reads
        // none of them), the full build's item list, and TT row lengths
        // marked unset
        CUDA_TRY(cudaMemcpyAsync(ctx->d_parts, hm.parts.data(), sizeof(gale::PartInfo) * NP, cudaMemcpyHostToDevice,
                                 ctx->stream));
        CUDA_TRY(cudaMemcpyAsync(ctx->d_all_items, ctx->all_items.data(), 4 * ctx->all_items.size(),
                                 cudaMemcpyHostToDevice, ctx->stream));
        CUDA_TRY(cudaMemsetAsync(ctx->d_tt_pos, 0xff, sizeof(int32_t) * std::max<int64_t>(1, hm.nt), ctx->stream));
    }
    CUDA_TRY(cudaMemcpyAsync(ctx->d_I_V, hm.I_V.data(), sizeof(int32_t) * (K + 1), cudaMemcpyHostToDevice,
                             ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(ctx->d_I_T, hm.I_T.data(), sizeof(int32_t) * (K + 1), cudaMemcpyHostToDevice,
                             ctx->stream));
    CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, 64, ctx->stream));
    gale_status st = plan_bins(ctx.get(), false);
    if (st == GALE_OK) st = upload_orders(ctx.get());
    if (st == GALE_OK) st = count_pass(ctx.get());
    // build plans: staging capacities from the exact sizes
    if (st == GALE_OK) st = plan_bins(ctx.get(), true);
    if (st == GALE_OK) st = upload_orders(ctx.get());
    if (st != GALE_OK) {
        std::string keep = gale::t_error;
        // A cluster cut into parts holds a triangle in three or more tets:
        // parts assume one partner per face, so the mesh loads again with no
        // cluster cut (the large ones then run whole, from global scratch,
        // with the general TT pass).
        const bool uncut = st == GALE_EDEVICE && ctx->last_err_word == gale::ERR_NONMANIFOLD && ctx->hm.NP > 0 &&
                           desc->part_vertices >= 0;
        gale_destroy(ctx.release());
        if (uncut) {
            gale_mesh_desc whole = *desc;
            whole.part_vertices = -1;
            return gale_load_mesh(&whole, out);
        }
        return fail(st, keep);
    }
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    // the host copy of the blocks is no longer needed
    hm.free_blocks();
    ctx->device_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = ctx.release();
    return GALE_OK;
}

gale_status gale_build_clusters(gale_ctx *ctx, const int32_t *ids, int32_t n, uint32_t mask, int32_t mode) {
    if (!ctx) return fail(GALE_EINVAL, "NULL context");
    if (ctx->device < 0) return fail(GALE_EINVAL, "host-only context");
    if (mask == 0 || (mask & ~ctx->precond))
        return fail(GALE_EINVAL, "mask must be a non-empty subset of the precondition mask");
    if (mode != GALE_MODE_PER_CLUSTER && mode != GALE_MODE_BATCHED) return fail(GALE_EINVAL, "unknown mode");
    std::lock_guard<std::mutex> lock(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->device));
    const int32_t K = ctx->hm.K;
    const bool all = (ids == nullptr || n <= 0);
    const int32_t cnt = all ? K : n;
    if (!all && n > K) return fail(GALE_EINVAL, "more ids than clusters");
    std::vector<int32_t> list(cnt);
    if (all) {
        std::iota(list.begin(), list.end(), 0);
    } else {
        std::vector<uint8_t> seen(K, 0);
        for (int32_t i = 0; i < n; ++i) {
            if (ids[i] < 0 || ids[i] >= K) return fail(GALE_EINVAL, "cluster id out of range");
            if (seen[ids[i]]++) return fail(GALE_EINVAL, "cluster id listed twice");
            list[i] = ids[i];
        }
    }
    // placement bookkeeping on the host (views); the device recomputes it
    ctx->bulk_offs.assign(size_t(cnt) * 10, 0);
    int64_t run[10] = {};
    for (int32_t i = 0; i < cnt; ++i) {
        int64_t L[10];
        gale::item_lengths(ctx, list[i], mask, L);
        for (int a = 0; a < 10; ++a) {
            ctx->bulk_offs[size_t(i) * 10 + a] = run[a];
            run[a] += L[a];
        }
    }
    gale_status st = ensure_bulk(ctx, run);
    if (st != GALE_OK) return st;
    for (int a = 0; a < 10; ++a) ctx->bulk_len[a] = run[a];
    ctx->bulk_ids = list;
    ctx->bulk_mask = mask;
    const gale::DevMesh dm = dev_mesh(ctx);
    const WorkItem *base = ctx->d_arrays_base + mask;
    int64_t launches = 0;
    if (mode == GALE_MODE_BATCHED && all) {
        cudaGraphExec_t &g = ctx->graphs[mask];
        if (!g) {
            cudaGraph_t graph;
            CUDA_TRY(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            int rc = gale::launch_bases(dm, ctx->hm.NP ? ctx->d_all_items : nullptr, int32_t(ctx->all_items.size()),
                                        ctx->d_sizes, mask, base, ctx->d_items, ctx->d_totals, ctx->d_bsum,
                                        ctx->stream);
            for (size_t b = 0; rc == 0 && b < ctx->bins.size(); ++b) {
                const gale::Bin &bin = ctx->bins[b];
                if (bin.cut) continue;  // its clusters' parts are in other bins
                rc = gale::launch_build(dm, bin.plan, ctx->d_items, ctx->d_order_all + ctx->order_all_off[b],
                                        int32_t(bin.clusters.size()), ctx->d_err, ctx->d_tickets + b,
                                        grid_of(bin, int32_t(bin.clusters.size())), ctx->stream, scratch_of(ctx, bin),
                                        plans_of(ctx, bin), bin.teams);
            }
            cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
            if (rc != 0) return cuda_fail(cudaError_t(rc), "capturing the batched build");
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
            ce = cudaGraphInstantiate(&g, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) {
                g = nullptr;
                return cuda_fail(ce, "cudaGraphInstantiate");
            }
        }
        CUDA_TRY(cudaGraphLaunch(g, ctx->stream));
        launches = 3;
        for (const auto &bin : ctx->bins) launches += !bin.cut;
    } else {
        // a partial batched build lists the parts of cut clusters in their place
        const std::vector<int32_t> items = mode == GALE_MODE_BATCHED ? expand_items(ctx, list) : list;
        const int32_t ni = int32_t(items.size());
        const int32_t *d_ids = nullptr;
        if (!all || ctx->hm.NP) {
            CUDA_TRY(cudaMemcpyAsync(ctx->d_ids, items.data(), size_t(ni) * 4, cudaMemcpyHostToDevice, ctx->stream));
            d_ids = ctx->d_ids;
        }
        int rc = gale::launch_bases(dm, d_ids, ni, ctx->d_sizes, mask, base, ctx->d_items, ctx->d_totals,
                                    ctx->d_bsum, ctx->stream);
        if (rc != 0) return cuda_fail(cudaError_t(rc), "bases launch");
        launches = 3;
        if (mode == GALE_MODE_PER_CLUSTER) {
            for (int32_t i = 0; i < cnt; ++i) {
                const gale::Bin &bin = ctx->bins[ctx->bin_of[list[i]]];
                rc = gale::launch_build_one(dm, bin.per_item ? ctx->h_plans[list[i]] : bin.plan, ctx->d_items, i,
                                            ctx->d_err, ctx->stream, scratch_of(ctx, bin));
                if (rc != 0) return cuda_fail(cudaError_t(rc), "per-cluster launch");
            }
            launches += cnt;
        } else {
            // partial batched build: per-bin item orders
            std::vector<int32_t> order;
            std::vector<std::vector<int64_t>> boff;
            if (!chunk_bin_orders(ctx, items, false, {0, ni}, order, boff))
                return fail(GALE_EINVAL, "a listed cluster is in no size bin");
            const std::vector<int64_t> &off = boff[0];
            CUDA_TRY(cudaMemcpyAsync(ctx->d_order_part, order.data(), order.size() * 4, cudaMemcpyHostToDevice,
                                     ctx->stream));
            for (size_t b = 0; b < ctx->bins.size(); ++b) {
                const int32_t nb = int32_t(off[b + 1] - off[b]);
                if (nb == 0) continue;
                const gale::Bin &bin = ctx->bins[b];
                rc = gale::launch_build(dm, bin.plan, ctx->d_items, ctx->d_order_part + off[b], nb, ctx->d_err,
                                        ctx->d_tickets + b, grid_of(bin, nb), ctx->stream, scratch_of(ctx, bin),
                                        plans_of(ctx, bin), bin.teams);
                if (rc != 0) return cuda_fail(cudaError_t(rc), "batched launch");
                ++launches;
            }
        }
    }
    ctx->last_launches = launches;
    return GALE_OK;
}

gale_status gale_synchronize(gale_ctx *ctx) {
    if (!ctx) return fail(GALE_EINVAL, "NULL context");
    if (ctx->device < 0) return GALE_OK;
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return check_device_error(ctx);
}

gale_status gale_bulk_view(gale_ctx *ctx, int32_t index, gale_view *out) {
    if (!ctx || !out) return fail(GALE_EINVAL, "NULL argument");
    if (index < 0 || index >= int32_t(ctx->bulk_ids.size())) return fail(GALE_ENOTFOUND, "no such bulk index");
    const int32_t k = ctx->bulk_ids[index];
    const int64_t *o = ctx->bulk_offs.data() + size_t(index) * 10;
    const uint32_t m = ctx->bulk_mask;
    memset(out, 0, sizeof(*out));
    out->cluster = k;
    out->mask = m;
    out->v_begin = ctx->hm.I_V[k];
    out->v_end = ctx->hm.I_V[k + 1];
    out->t_begin = ctx->hm.I_T[k];
    out->t_end = ctx->hm.I_T[k + 1];
    out->n_edges = int32_t(ctx->sizes[size_t(5) * k + 2]);
    const int32_t *const *b = ctx->bulk;
    if (m & GALE_VT) { out->vt_off = b[0] + o[0]; out->vt_val = b[1] + o[1]; }
    if (m & GALE_VV) { out->vv_off = b[2] + o[2]; out->vv_val = b[3] + o[3]; }
    if (m & GALE_ET) {
        out->et_uoff = b[4] + o[4]; out->et_w = b[5] + o[5]; out->et_off = b[6] + o[6]; out->et_val = b[7] + o[7];
    }
    if (m & GALE_TT) { out->tt_off = b[8] + o[8]; out->tt_val = b[9] + o[9]; }
    return GALE_OK;
}

gale_status gale_bulk_arrays(gale_ctx *ctx, gale_arrays *dev, int64_t *lengths) {
    if (!ctx) return fail(GALE_EINVAL, "NULL context");
    if (dev) {
        int32_t **d = &dev->vt_off;
        for (int a = 0; a < 10; ++a) d[a] = ctx->bulk[a];
    }
    if (lengths)
        for (int a = 0; a < 10; ++a) lengths[a] = ctx->bulk_len[a];
    return GALE_OK;
}

gale_status gale_bulk_export(gale_ctx *ctx, uint32_t mask, const gale_arrays *host_dst) {
    if (!ctx || !host_dst) return fail(GALE_EINVAL, "NULL argument");
    if (ctx->device < 0) return fail(GALE_EINVAL, "host-only context");
    CUDA_TRY(cudaSetDevice(ctx->device));
    int32_t *const *h = &host_dst->vt_off;
    const uint32_t rel_of[10] = {GALE_VT, GALE_VT, GALE_VV, GALE_VV, GALE_ET, GALE_ET, GALE_ET, GALE_ET, GALE_TT, GALE_TT};
    for (int a = 0; a < 10; ++a) {
        if (!(mask & rel_of[a] & ctx->bulk_mask) || ctx->bulk_len[a] == 0) continue;
        if (!h[a]) return fail(GALE_EINVAL, "NULL host buffer for a requested array");
        const gale_status st = gale::copy_to_host(ctx, h[a], ctx->bulk[a], size_t(ctx->bulk_len[a]) * 4);
        if (st != GALE_OK) return st;
    }
    return GALE_OK;
}

gale_status gale_copy_to_host(gale_ctx *ctx, void *dst, const void *src, size_t bytes) {
    if (!ctx || (bytes > 0 && (!dst || !src))) return fail(GALE_EINVAL, "NULL argument");
    if (ctx->device < 0) return fail(GALE_EINVAL, "host-only context");
    CUDA_TRY(cudaSetDevice(ctx->device));
    return gale::copy_to_host(ctx, dst, src, bytes);
}

gale_status gale_build_export(gale_ctx *ctx, const int32_t *ids, int32_t n, uint32_t mask,
                              const gale_arrays *host_dst, int32_t chunks) {
    if (!ctx || !host_dst) return fail(GALE_EINVAL, "NULL argument");
    if (ctx->device < 0) return fail(GALE_EINVAL, "host-only context");
    if (mask == 0 || (mask & ~ctx->precond))
        return fail(GALE_EINVAL, "mask must be a non-empty subset of the precondition mask");
    if (chunks < 0 || chunks > kMaxExportChunks)
        return fail(GALE_EINVAL, "chunks must be 0 (automatic) to " + std::to_string(kMaxExportChunks));
    std::lock_guard<std::mutex> lock(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->device));
    const int32_t K = ctx->hm.K;
    const bool all = (ids == nullptr || n <= 0);
    const int32_t cnt = all ? K : n;
    if (!all && n > K) return fail(GALE_EINVAL, "more ids than clusters");
    std::vector<int32_t> list(cnt);
    if (all) {
        std::iota(list.begin(), list.end(), 0);
    } else {
        std::vector<uint8_t> seen(K, 0);
        for (int32_t i = 0; i < cnt; ++i) {
            if (ids[i] < 0 || ids[i] >= K) return fail(GALE_EINVAL, "cluster id out of range");
            if (seen[ids[i]]++) return fail(GALE_EINVAL, "cluster id listed twice");
            list[i] = ids[i];
        }
    }
    int32_t *const *h = &host_dst->vt_off;
    const uint32_t rel_of[10] = {GALE_VT, GALE_VT, GALE_VV, GALE_VV, GALE_ET, GALE_ET, GALE_ET, GALE_ET, GALE_TT, GALE_TT};
    for (int a = 0; a < 10; ++a)
        if ((mask & rel_of[a]) && !h[a]) return fail(GALE_EINVAL, "NULL host buffer for a requested array");
    // placement of every listed cluster, and the chunk boundaries: about
    // equal output bytes per chunk
    ctx->bulk_offs.assign(size_t(cnt) * 10, 0);
    int64_t run[10] = {};
    std::vector<int64_t> bytes_before(size_t(cnt) + 1, 0);
    for (int32_t i = 0; i < cnt; ++i) {
        int64_t L[10];
        gale::item_lengths(ctx, list[i], mask, L);
        int64_t b = 0;
        for (int a = 0; a < 10; ++a) {
            ctx->bulk_offs[size_t(i) * 10 + a] = run[a];
            run[a] += L[a];
            b += 4 * L[a];
        }
        bytes_before[i + 1] = bytes_before[i] + b;
    }
    gale_status st = ensure_bulk(ctx, run);
    if (st != GALE_OK) return st;
    for (int a = 0; a < 10; ++a) ctx->bulk_len[a] = run[a];
    ctx->bulk_ids = list;
    ctx->bulk_mask = mask;
    // automatic: one chunk per 256 MB of output, at most 16 (measured at
    // 256^3: 16 chunks 44.4 ms, 8 chunks 44.8 ms, 4 chunks 45.7 ms)
    if (chunks == 0) chunks = int32_t(std::min<int64_t>(16, std::max<int64_t>(1, bytes_before[cnt] >> 28)));
    chunks = std::max(1, std::min(chunks, cnt));
    std::vector<int32_t> cut(size_t(chunks) + 1, cnt);
    cut[0] = 0;
    for (int32_t c = 1; c < chunks; ++c) {
        const int64_t target = bytes_before[cnt] * c / chunks;
        cut[c] = int32_t(std::lower_bound(bytes_before.begin(), bytes_before.end(), target) - bytes_before.begin());
        cut[c] = std::max(cut[c], cut[c - 1]);
    }
    if (!ctx->copy_stream) CUDA_TRY(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    while (int32_t(ctx->chunk_events.size()) < kMaxExportChunks) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->chunk_events.push_back(e);
    }
    if (!ctx->d_chunk_base) {
        ctx->d_chunk_base = static_cast<WorkItem *>(ctx->dalloc(sizeof(WorkItem) * kMaxExportChunks));
        if (!ctx->d_chunk_base) return fail(GALE_ENOMEM, "device allocation failed");
    }
    // per chunk: base pointers shifted to the chunk's first element, and the
    // chunk's items (cut clusters replaced by their parts) grouped by size
    // bin (largest working set first)
    std::vector<WorkItem> cbase(chunks);
    std::vector<int32_t> order;
    std::vector<std::vector<int64_t>> boff;
    std::vector<int32_t> items = expand_items(ctx, list);
    std::vector<int32_t> icut(cut);  // chunk boundaries in the item list
    if (ctx->hm.NP) {
        std::vector<int32_t> first(size_t(cnt) + 1, 0);  // item position of each listed cluster
        for (int32_t i = 0; i < cnt; ++i) {
            const int32_t k = list[i];
            const int32_t np = ctx->hm.part_first[k + 1] - ctx->hm.part_first[k];
            first[i + 1] = first[i] + std::max(np, 1);
        }
        for (auto &c : icut) c = first[c];
    }
    const int32_t ni = int32_t(items.size());
    if (!chunk_bin_orders(ctx, items, all && ctx->hm.NP == 0, icut, order, boff))
        return fail(GALE_EINVAL, "a listed cluster is in no size bin");
    for (int32_t c = 0; c < chunks; ++c) {
        const int32_t i0 = cut[c];
        int32_t *ptr[10];
        for (int a = 0; a < 10; ++a) {
            const int64_t off = i0 < cnt ? ctx->bulk_offs[size_t(i0) * 10 + a] : run[a];
            ptr[a] = (mask & rel_of[a]) ? ctx->bulk[a] + off : nullptr;
        }
        WorkItem &w = cbase[c];
        memset(&w, 0, sizeof(w));
        w.vt_off = ptr[0]; w.vt_val = ptr[1]; w.vv_off = ptr[2]; w.vv_val = ptr[3];
        w.eu_off = ptr[4]; w.e_w = ptr[5]; w.et_off = ptr[6]; w.et_val = ptr[7];
        w.tt_off = ptr[8]; w.tt_val = ptr[9];
    }
    CUDA_TRY(cudaMemcpyAsync(ctx->d_ids, items.data(), size_t(ni) * 4, cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(ctx->d_order_part, order.data(), order.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(cudaMemcpyAsync(ctx->d_chunk_base, cbase.data(), sizeof(WorkItem) * chunks, cudaMemcpyHostToDevice,
                             ctx->stream));
    const gale::DevMesh dm = dev_mesh(ctx);
    int64_t launches = 0;
    for (int32_t c = 0; c < chunks; ++c) {
        const int32_t i0 = cut[c];
        const int32_t j0 = icut[c], nc = icut[c + 1] - j0;
        if (nc > 0) {
            int rc = gale::launch_bases(dm, ctx->d_ids + j0, nc, ctx->d_sizes, mask, ctx->d_chunk_base + c,
                                        ctx->d_items + j0, ctx->d_totals, ctx->d_bsum, ctx->stream);
            if (rc != 0) return cuda_fail(cudaError_t(rc), "bases launch");
            launches += 3;
            for (size_t b = 0; b < ctx->bins.size(); ++b) {
                const int32_t nb = int32_t(boff[c][b + 1] - boff[c][b]);
                if (nb == 0) continue;
                const gale::Bin &bin = ctx->bins[b];
                rc = gale::launch_build(dm, bin.plan, ctx->d_items + j0, ctx->d_order_part + boff[c][b], nb,
                                        ctx->d_err, ctx->d_tickets + b, grid_of(bin, nb), ctx->stream,
                                        scratch_of(ctx, bin), plans_of(ctx, bin), bin.teams);
                if (rc != 0) return cuda_fail(cudaError_t(rc), "batched launch");
                ++launches;
            }
        }
        // the chunk's outputs leave while the next chunk builds
        CUDA_TRY(cudaEventRecord(ctx->chunk_events[c], ctx->stream));
        CUDA_TRY(cudaStreamWaitEvent(ctx->copy_stream, ctx->chunk_events[c], 0));
        for (int a = 0; a < 10; ++a) {
            if (!(mask & rel_of[a])) continue;
            const int64_t o0 = i0 < cnt ? ctx->bulk_offs[size_t(i0) * 10 + a] : run[a];
            const int64_t o1 = cut[c + 1] < cnt ? ctx->bulk_offs[size_t(cut[c + 1]) * 10 + a] : run[a];
            if (o1 > o0)
                CUDA_TRY(cudaMemcpyAsync(h[a] + o0, ctx->bulk[a] + o0, size_t(o1 - o0) * 4, cudaMemcpyDeviceToHost,
                                         ctx->copy_stream));
        }
    }
    ctx->last_launches = launches;
    CUDA_TRY(cudaStreamSynchronize(ctx->copy_stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
}

gale_status gale_get_permutations(gale_ctx *ctx, int32_t *vperm, int32_t *tperm) {
    if (!ctx) return fail(GALE_EINVAL, "NULL context");
    if (vperm) memcpy(vperm, ctx->hm.vperm.data(), sizeof(int32_t) * ctx->hm.nv);
    if (tperm) memcpy(tperm, ctx->hm.tperm.data(), sizeof(int32_t) * ctx->hm.nt);
    return GALE_OK;
}

gale_status gale_get_intervals(gale_ctx *ctx, int64_t *I_V, int64_t *I_T, int64_t *sizes) {
    if (!ctx) return fail(GALE_EINVAL, "NULL context");
    const int32_t K = ctx->hm.K;
    for (int32_t k = 0; k <= K; ++k) {
        if (I_V) I_V[k] = ctx->hm.I_V[k];
        if (I_T) I_T[k] = ctx->hm.I_T[k];
    }
    if (sizes) {
        if (ctx->sizes.empty()) memset(sizes, 0, sizeof(int64_t) * 5 * K);
        else memcpy(sizes, ctx->sizes.data(), sizeof(int64_t) * 5 * K);
    }
    return GALE_OK;
}

gale_status gale_get_rows(gale_ctx *ctx, int32_t *rows) {
    if (!ctx || !rows) return fail(GALE_EINVAL, "NULL argument");
    gale::parallel_copy(rows, ctx->hm.rows.data(), 4 * ctx->hm.nt, gale::host_threads(0));
    return GALE_OK;
}

gale_status gale_get_working_set(gale_ctx *ctx, int32_t k, int32_t *ext, int64_t *n_ext, int32_t *halo,
                                 int64_t *n_halo) {
    if (!ctx || !n_ext || !n_halo) return fail(GALE_EINVAL, "NULL argument");
    if (k < 0 || k >= ctx->hm.K) return fail(GALE_ENOTFOUND, "no such cluster");
    const auto &hm = ctx->hm;
    const int64_t ne = hm.ext_off[k + 1] - hm.ext_off[k], nh = hm.halo_off[k + 1] - hm.halo_off[k];
    if (*n_ext < ne || *n_halo < nh) {
        *n_ext = ne;
        *n_halo = nh;
        return fail(GALE_EINVAL, "buffers too small");
    }
    if (ext) memcpy(ext, hm.ext.data() + hm.ext_off[k], sizeof(int32_t) * ne);
    if (halo) memcpy(halo, hm.halo.data() + hm.halo_off[k], sizeof(int32_t) * nh);
    *n_ext = ne;
    *n_halo = nh;
    return GALE_OK;
}

gale_status gale_get_info(gale_ctx *ctx, gale_info *out) {
    if (!ctx || !out) return fail(GALE_EINVAL, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->nv = ctx->hm.nv;
    out->nt = ctx->hm.nt;
    out->nclusters = ctx->hm.K;
    out->device = ctx->device;
    out->n_edges = ctx->totals[2];
    for (int a = 0; a < 5; ++a) out->total[a] = ctx->totals[a];
    out->block_bytes = ctx->hm.blocks_words * 4;
    out->ext_tets = ctx->hm.ext_total;
    out->halo_tets = ctx->hm.halo_total;
    out->nbins = int32_t(ctx->bins.size());
    int32_t mx = 0;
    for (int32_t k = 0; k < ctx->hm.K; ++k) {
        const gale::ClusterStat &s = ctx->hm.stats[k];
        mx = std::max(mx, s.n_ext + s.n_own + s.n_halo);
    }
    out->max_cluster_tets = mx;
    out->load_host_seconds = ctx->hm.host_seconds;
    out->load_device_seconds = ctx->device_seconds;
    out->nparts = ctx->hm.NP;
    int32_t cut = 0;
    for (int32_t k = 0; k < ctx->hm.K; ++k) cut += ctx->hm.part_first[k + 1] > ctx->hm.part_first[k];
    out->cut_clusters = cut;
    return GALE_OK;
}

gale_status gale_set_tuning(gale_ctx *ctx, int32_t threads, int32_t ctas_per_sm) {
    if (!ctx) return fail(GALE_EINVAL, "NULL context");
    if (threads != 0 && (threads < 64 || threads > 1024 || threads % 32 != 0))
        return fail(GALE_EINVAL, "threads must be 0 or a multiple of 32 in [64, 1024]");
    if (ctx->device < 0) return GALE_OK;
    std::lock_guard<std::mutex> lock(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    ctx->threads_override = threads;
    ctx->ctas_override = ctas_per_sm;
    gale_status st = plan_bins(ctx, true);
    if (st != GALE_OK) return st;
    st = upload_orders(ctx);
    for (auto &g : ctx->graphs)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return st;
}

gale_status gale_set_teams(gale_ctx *ctx, int32_t team_threads, int32_t teams) {
    if (!ctx) return fail(GALE_EINVAL, "NULL context");
    if (teams != 0 && (teams < 2 || teams > 15 || team_threads < 32 || team_threads % 32 != 0 ||
                       team_threads * teams > 512))
        return fail(GALE_EINVAL, "teams must be 0, or 2..15 teams of a multiple of 32 threads, at most 512 in all");
    if (ctx->device < 0) return GALE_OK;
    std::lock_guard<std::mutex> lock(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    const int smem_limit = gale::dynamic_smem_limit();
    int max_total = 0;
    for (auto &b : ctx->bins) {
        if (!team_eligible(ctx, b)) continue;
        if (teams == 0) {
            b.teams = 0;
            continue;
        }
        const gale::SmemPlan p = gale::plan_smem(b.plan.caps, team_threads);
        if (int64_t(p.total) * teams > smem_limit) continue;
        max_total = std::max(max_total, p.total * teams);
        if (!gale::prepare_kernels(max_total)) return fail(GALE_ECUDA, "setting the kernels' shared memory limit failed");
        const int per = gale::max_ctas_per_sm_teams(p, teams);
        if (per < 1) continue;
        b.plan = p;
        b.teams = teams;
        b.ctas_per_sm = per;
        b.grid = std::max(1, per * ctx->sm_count);
    }
    for (auto &g : ctx->graphs)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return GALE_OK;
}

gale_status gale_get_bin_members(gale_ctx *ctx, int32_t *out) {
    if (!ctx || !out) return fail(GALE_EINVAL, "NULL argument");
    size_t w = 0;
    for (const auto &b : ctx->bins)
        for (int32_t k : b.clusters) out[w++] = k;
    return GALE_OK;
}

gale_status gale_autotune(gale_ctx *ctx, uint32_t mask, int32_t reps, float *best_ms, int32_t max_bins) {
    if (!ctx) return fail(GALE_EINVAL, "NULL context");
    if (ctx->device < 0) return fail(GALE_EINVAL, "host-only context");
    if (mask == 0 || (mask & ~ctx->precond))
        return fail(GALE_EINVAL, "mask must be a non-empty subset of the precondition mask");
    if (reps < 0) return fail(GALE_EINVAL, "reps must be >= 0");
    if (reps == 0) reps = 2;
    std::lock_guard<std::mutex> lock(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->device));
    const int32_t K = ctx->hm.K;
    // outputs of every cluster: one placement pass, then bins are timed alone
    int64_t run[10] = {};
    ctx->bulk_offs.assign(size_t(K) * 10, 0);
    for (int32_t k = 0; k < K; ++k) {
        int64_t L[10];
        gale::item_lengths(ctx, k, mask, L);
        for (int a = 0; a < 10; ++a) {
            ctx->bulk_offs[size_t(k) * 10 + a] = run[a];
            run[a] += L[a];
        }
    }
    gale_status st = ensure_bulk(ctx, run);
    if (st != GALE_OK) return st;
    for (int a = 0; a < 10; ++a) ctx->bulk_len[a] = run[a];
    ctx->bulk_ids.resize(K);
    std::iota(ctx->bulk_ids.begin(), ctx->bulk_ids.end(), 0);
    ctx->bulk_mask = mask;
    const gale::DevMesh dm = dev_mesh(ctx);
    int rc = gale::launch_bases(dm, ctx->hm.NP ? ctx->d_all_items : nullptr, int32_t(ctx->all_items.size()),
                                ctx->d_sizes, mask, ctx->d_arrays_base + mask, ctx->d_items, ctx->d_totals,
                                ctx->d_bsum, ctx->stream);
    if (rc != 0) return cuda_fail(cudaError_t(rc), "bases launch");
    const int smem_limit = gale::dynamic_smem_limit();
    if (!gale::prepare_kernels(smem_limit)) return fail(GALE_ECUDA, "setting the kernels' shared memory limit failed");
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    const int cand_threads[] = {128, 256, 384, 512, 768, 1024};
    for (size_t b = 0; b < ctx->bins.size(); ++b) {
        gale::Bin &bin = ctx->bins[b];
        const int32_t nb = int32_t(bin.clusters.size());
        if (bin.cut) {  // batched builds run these clusters' parts instead
            if (best_ms && int32_t(b) < max_bins) best_ms[b] = 0.f;
            continue;
        }
        float best = -1.f;
        gale::SmemPlan best_plan = bin.plan;
        int best_grid = bin.grid, best_per = bin.ctas_per_sm;
        std::vector<gale::SmemPlan> best_members;
        for (int T : cand_threads) {
            gale::SmemPlan plan = gale::plan_smem(bin.plan.caps, T);
            if (bin.per_item) {
                // the members' own plans at this block size; the envelope
                // takes the largest shared memory
                int top = 0;
                for (int32_t k : bin.clusters) {
                    ctx->h_plans[k] = gale::plan_smem(bin_caps(ctx, k), T);
                    top = std::max(top, ctx->h_plans[k].total);
                }
                plan.threads = T;
                plan.total = top;
                CUDA_TRY(cudaStreamSynchronize(ctx->stream));
                CUDA_TRY(cudaMemcpy(ctx->d_plans, ctx->h_plans.data(), sizeof(gale::SmemPlan) * ctx->h_plans.size(),
                                    cudaMemcpyHostToDevice));
            }
            if (!bin.spill && plan.total > smem_limit) continue;
            int max_per = gale::max_ctas_per_sm(plan, bin.spill, bin.per_item);
            if (bin.spill) max_per = std::min(max_per, 2);
            // persistent grids of 1 .. max_per CTAs per SM; a global-scratch
            // bin also tries a half and a quarter of the SMs, whose scratch
            // may stay in L2
            std::vector<std::pair<int, int>> cands;  // (CTAs per SM, grid)
            for (int per = 1; per <= max_per; ++per) cands.push_back({per, per * ctx->sm_count});
            if (bin.spill && max_per >= 1)
                for (int div : {2, 4}) cands.push_back({1, std::max(1, ctx->sm_count / div)});
            for (const auto &pc : cands) {
                const int per = pc.first;
                const int grid = std::max(1, std::min<int>(nb, pc.second));
                char *scratch = nullptr;
                if (bin.spill) {
                    const int64_t need = int64_t(grid) * plan.total;
                    if (need > ctx->spill_bytes) {
                        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
                        if (ctx->d_spill) ctx->dfree(ctx->d_spill);
                        ctx->d_spill = static_cast<char *>(ctx->dalloc(size_t(need)));
                        ctx->spill_bytes = ctx->d_spill ? need : 0;
                        if (!ctx->d_spill) {
                            cudaEventDestroy(e0);
                            cudaEventDestroy(e1);
                            return fail(GALE_ENOMEM, "device allocation of the large-cluster scratch failed");
                        }
                    }
                    scratch = ctx->d_spill;
                }
                auto launch = [&]() {
                    return gale::launch_build(dm, plan, ctx->d_items, ctx->d_order_all + ctx->order_all_off[b], nb,
                                              ctx->d_err, ctx->d_tickets + b, grid, ctx->stream, scratch,
                                              plans_of(ctx, bin));
                };
                rc = launch();
                CUDA_TRY(cudaEventRecord(e0, ctx->stream));
                for (int r = 0; rc == 0 && r < reps; ++r) rc = launch();
                CUDA_TRY(cudaEventRecord(e1, ctx->stream));
                if (rc != 0) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return cuda_fail(cudaError_t(rc), "autotune launch");
                }
                CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                ms /= float(reps);
                if (best < 0.f || ms < best) {
                    best = ms;
                    best_plan = plan;
                    best_grid = grid;
                    best_per = per;
                    if (bin.per_item) {
                        best_members.clear();
                        for (int32_t k : bin.clusters) best_members.push_back(ctx->h_plans[k]);
                    }
                }
            }
        }
        // several clusters per CTA, one team of T threads each
        int best_teams = 0;
        if (team_eligible(ctx, bin)) {
            for (int T : {32, 64, 128})
                for (int tm : {2, 4, 8}) {
                    if (T * tm > 512) continue;
                    const gale::SmemPlan plan = gale::plan_smem(bin.plan.caps, T);
                    if (int64_t(plan.total) * tm > smem_limit) continue;
                    const int per = gale::max_ctas_per_sm_teams(plan, tm);
                    if (per < 1) continue;
                    gale::Bin probe;
                    probe.teams = tm;
                    probe.grid = per * ctx->sm_count;
                    const int grid = grid_of(probe, nb);
                    auto launch = [&]() {
                        return gale::launch_build(dm, plan, ctx->d_items, ctx->d_order_all + ctx->order_all_off[b],
                                                  nb, ctx->d_err, ctx->d_tickets + b, grid, ctx->stream, nullptr,
                                                  nullptr, tm);
                    };
                    rc = launch();
                    CUDA_TRY(cudaEventRecord(e0, ctx->stream));
                    for (int r = 0; rc == 0 && r < reps; ++r) rc = launch();
                    CUDA_TRY(cudaEventRecord(e1, ctx->stream));
                    if (rc != 0) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return cuda_fail(cudaError_t(rc), "autotune launch");
                    }
                    CUDA_TRY(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                    ms /= float(reps);
                    if (best < 0.f || ms < best) {
                        best = ms;
                        best_plan = plan;
                        best_grid = probe.grid;
                        best_per = per;
                        best_teams = tm;
                    }
                }
        }
        if (best >= 0.f) {
            bin.plan = best_plan;
            bin.grid = best_grid;
            bin.ctas_per_sm = best_per;
            bin.teams = best_teams;
        }
        if (bin.per_item && !best_members.empty()) {
            for (size_t i = 0; i < bin.clusters.size(); ++i) ctx->h_plans[bin.clusters[i]] = best_members[i];
            CUDA_TRY(cudaStreamSynchronize(ctx->stream));
            CUDA_TRY(cudaMemcpy(ctx->d_plans, ctx->h_plans.data(), sizeof(gale::SmemPlan) * ctx->h_plans.size(),
                                cudaMemcpyHostToDevice));
        }
        if (best_ms && int32_t(b) < max_bins) best_ms[b] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int max_total = 0;
    for (auto &bin : ctx->bins)
        if (!bin.spill) max_total = std::max(max_total, bin.plan.total * std::max(1, bin.teams));
    gale::prepare_kernels(max_total);
    for (auto &g : ctx->graphs)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    st = check_device_error(ctx);
    return st;
}

gale_status gale_get_bins(gale_ctx *ctx, int32_t *out, int32_t max_bins, int32_t *nbins) {
    if (!ctx || !nbins) return fail(GALE_EINVAL, "NULL argument");
    *nbins = int32_t(ctx->bins.size());
    for (int32_t b = 0; b < *nbins && b < max_bins && out; ++b) {
        const gale::Bin &bin = ctx->bins[b];
        int32_t *o = out + 9 * b;
        o[0] = int32_t(bin.clusters.size());
        o[1] = bin.plan.threads;
        o[2] = bin.plan.total;
        o[3] = bin.ctas_per_sm;
        o[4] = bin.grid;
        o[5] = bin.spill ? 1 : 0;
        o[6] = bin.per_item ? 1 : 0;
        int32_t parts = 0;
        for (int32_t k : bin.clusters) parts += k >= ctx->hm.K;
        o[7] = bin.cut ? -1 : parts;
        o[8] = bin.teams;
    }
    return GALE_OK;
}

void *gale_stream(gale_ctx *ctx) { return ctx ? static_cast<void *>(ctx->stream) : nullptr; }

int64_t gale_last_launch_count(gale_ctx *ctx) { return ctx ? ctx->last_launches : 0; }

}  // extern "C"
