// Allocation-free batched build (gale_build_clusters_noalloc).
//
// Some callers cannot call cudaMalloc at the point where they need
// relations: a serving thread that must not synchronise the device (cudaMalloc
// and cudaFree can), an application that hands all of HBM to its own pool up
// front, or code that runs where allocation is forbidden.  This entry point
// builds into device arrays the caller already owns, and keeps every piece of
// scratch the batched build needs - the work items, the cluster and per-bin
// order lists, the persistent-grid ticket counters and the device error word -
// in one fixed array in device global memory that every GPU which loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "gale_ctx.h"

namespace {

constexpr int32_t kNoAllocMaxClusters = 4096;  // clusters per call
constexpr int32_t kNoAllocMaxBins = 32;        // size bins of the context
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    gale::WorkItem items[kNoAllocMaxClusters];
    gale::WorkItem base;  // the caller's ten output base pointers
    int32_t ids[kNoAllocMaxClusters];
    int32_t order[kNoAllocMaxClusters];
    int32_t tickets[kNoAllocMaxBins];
    int32_t err;
    int32_t pad;
    int64_t totals[16];
    int64_t bsum[(kNoAllocMaxClusters + 255) / 256 * 10 + 16];  // output placement block sums
};

// The scratch: ~430 KB of device global memory, shared by every call.  Host
// code must not pass &g_noalloc to a kernel (it is a host-side stand-in for
// the device symbol); it uses the address cudaGetSymbolAddress returns.
static __device__ __align__(256) NoAllocScratch g_noalloc;

NoAllocScratch *g_addr[kMaxDevices] = {};  // device address of g_noalloc, per device
std::mutex g_setup_mu;                      // guards the one-time address lookup

gale_status fail(gale_status s, const std::string &msg) {
    gale::set_error(msg);
    return s;
}

}  // namespace

extern "C" gale_status gale_build_clusters_noalloc(gale_ctx *ctx, const int32_t *ids, int32_t n, uint32_t mask,
                                                   const gale_arrays *dev_out, const int64_t *lengths) {
    if (!ctx || !ids || !dev_out || !lengths) return fail(GALE_EINVAL, "NULL argument");
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return fail(GALE_EINVAL, "not a device context");
    if (mask == 0 || (mask & ~ctx->precond))
        return fail(GALE_EINVAL, "mask must be a non-empty subset of the precondition mask");
    if (n < 1 || n > kNoAllocMaxClusters)
        return fail(GALE_EINVAL, "gale_build_clusters_noalloc takes 1 to " + std::to_string(kNoAllocMaxClusters) +
                                     " clusters per call, got " + std::to_string(n));
    if (int32_t(ctx->bins.size()) > kNoAllocMaxBins)
        return fail(GALE_EINVAL, "the context has more than " + std::to_string(kNoAllocMaxBins) + " size bins");
    const int32_t K = ctx->hm.K;
    for (int32_t i = 0; i < n; ++i) {
        if (ids[i] < 0 || ids[i] >= K) return fail(GALE_EINVAL, "cluster id out of range");
        if (ctx->bins[ctx->bin_of[ids[i]]].spill)
            return fail(GALE_EINVAL, "cluster " + std::to_string(ids[i]) +
                                         " is too large for shared memory; the allocation-free build takes only "
                                         "clusters that fit");
    }
    int32_t *const *out = &dev_out->vt_off;
    const uint32_t rel_of[10] = {GALE_VT, GALE_VT, GALE_VV, GALE_VV, GALE_ET, GALE_ET, GALE_ET, GALE_ET, GALE_TT, GALE_TT};
    for (int a = 0; a < 10; ++a)
        if ((mask & rel_of[a]) && !out[a]) return fail(GALE_EINVAL, "NULL device array for a requested relation");
    // every requested array must hold the list's output: the kernels place
    // each cluster at its offset in the caller's arrays without bounds
    {
        static const char *names[10] = {"vt_off", "vt_val", "vv_off", "vv_val", "et_uoff",
                                        "et_w",   "et_off", "et_val", "tt_off", "tt_val"};
        int64_t need[10] = {};
        for (int32_t i = 0; i < n; ++i) {
            int64_t L[10];
            gale::item_lengths(ctx, ids[i], mask, L);
            for (int a = 0; a < 10; ++a) need[a] += L[a];
        }
        for (int a = 0; a < 10; ++a)
            if ((mask & rel_of[a]) && lengths[a] < need[a])
                return fail(GALE_EINVAL, std::string("device array ") + names[a] + " holds " +
                                             std::to_string(lengths[a]) + " elements, the list needs " +
                                             std::to_string(need[a]));
    }

    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail(GALE_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    NoAllocScratch *S;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> g(g_setup_mu);
        if (!g_addr[ctx->device]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc);
            if (e != cudaSuccess || !p)
                return fail(GALE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_addr[ctx->device] = static_cast<NoAllocScratch *>(p);
        }
        S = g_addr[ctx->device];
    }
    // work order: items grouped by size bin (staged on this call's stack;
    // the copy below has consumed it before the call returns)
    int32_t order[kNoAllocMaxClusters];
    int32_t cnt[kNoAllocMaxBins + 1] = {};
    const int32_t nb = int32_t(ctx->bins.size());
    for (int32_t i = 0; i < n; ++i) cnt[ctx->bin_of[ids[i]] + 1]++;
    for (int32_t b = 0; b < nb; ++b) cnt[b + 1] += cnt[b];
    int32_t cur[kNoAllocMaxBins];
    for (int32_t b = 0; b < nb; ++b) cur[b] = cnt[b];
    for (int32_t i = 0; i < n; ++i) order[cur[ctx->bin_of[ids[i]]]++] = i;

    gale::WorkItem base;
    memset(&base, 0, sizeof(base));
    base.vt_off = (mask & GALE_VT) ? out[0] : nullptr;
    base.vt_val = (mask & GALE_VT) ? out[1] : nullptr;
    base.vv_off = (mask & GALE_VV) ? out[2] : nullptr;
    base.vv_val = (mask & GALE_VV) ? out[3] : nullptr;
    base.eu_off = (mask & GALE_ET) ? out[4] : nullptr;
    base.e_w = (mask & GALE_ET) ? out[5] : nullptr;
    base.et_off = (mask & GALE_ET) ? out[6] : nullptr;
    base.et_val = (mask & GALE_ET) ? out[7] : nullptr;
    base.tt_off = (mask & GALE_TT) ? out[8] : nullptr;
    base.tt_val = (mask & GALE_TT) ? out[9] : nullptr;

    cudaStream_t s = ctx->stream;
    // the scratch keeps the previous call's contents: the error word must
    // start at zero (ticket counters are reset by each launch)
    if ((e = cudaMemsetAsync(&S->err, 0, sizeof(int32_t), s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(S->ids, ids, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(S->order, order, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(&S->base, &base, sizeof(base), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(GALE_ECUDA, std::string("staging the work list: ") + cudaGetErrorString(e));
    const gale::DevMesh dm{ctx->d_blocks, ctx->d_blk_off, ctx->d_I_V, ctx->d_I_T, K};
    if (gale::bases_scratch_words(n) > int(sizeof(S->bsum) / sizeof(int64_t)))
        return fail(GALE_EINVAL, "placement scratch too small");
    int rc = gale::launch_bases(dm, S->ids, n, ctx->d_sizes, mask, &S->base, S->items, S->totals, S->bsum, s);
    for (int32_t b = 0; rc == 0 && b < nb; ++b) {
        const int32_t m = cnt[b + 1] - cnt[b];
        if (m == 0) continue;
        const gale::Bin &bin = ctx->bins[b];
        rc = gale::launch_build(dm, bin.plan, S->items, S->order + cnt[b], m, &S->err, &S->tickets[b],
                                bin.grid < m ? bin.grid : m, s, nullptr, bin.per_item ? ctx->d_plans : nullptr);
    }
    if (rc != 0) return fail(GALE_ECUDA, std::string("launch: ") + cudaGetErrorString(cudaError_t(rc)));
    int32_t err = 0;
    if ((e = cudaMemcpyAsync(&err, &S->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(GALE_ECUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
    if (err) return fail(GALE_EDEVICE, "kernel error word " + std::to_string(err));
    return GALE_OK;
}
