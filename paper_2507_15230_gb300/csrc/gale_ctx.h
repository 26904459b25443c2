// The context behind the opaque gale_ctx handle (internal).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "gale_host.h"

namespace gale {

struct Serve;        // serving loop state (gale_serve.cpp)
struct Enumeration;  // edge / triangle lists (gale_enum.cpp)
struct Cobound;      // coboundary pass device state (gale_cobound.cu)

struct Bin {
    SmemPlan plan;
    std::vector<int32_t> clusters;  // members, largest working set first
    int grid = 0;                   // persistent CTAs
    int ctas_per_sm = 0;
    bool spill = false;             // regions in global scratch (working set too large for shared memory)
    bool per_item = false;          // each member runs under its own plan (gale_ctx::d_plans); `plan` is the
                                    // launch envelope: block size and the largest member's shared memory
    bool cut = false;               // members are clusters cut into parts: batched builds run the parts
                                    // (items K..K+NP-1, in other bins) instead; the other forms use this bin
    int teams = 0;                  // > 0: batched builds run `teams` clusters per CTA at once, one team of
                                    // plan.threads threads each (the other forms run one per CTA)
    bool tt_general = false;        // members are non-manifold clusters: their TT rows take the general
                                    // pass, which the per-item and global-scratch kernels carry
};

struct DevAlloc {
    void *ptr = nullptr;
    size_t bytes = 0;
};

void set_error(const std::string &msg);

}  // namespace gale

struct gale_ctx {
    gale::HostMesh hm;
    uint32_t precond = 0;
    int device = -1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    gale_alloc_fn alloc_fn = nullptr;
    gale_free_fn free_fn = nullptr;
    void *alloc_ctx = nullptr;
    int64_t cache_budget = 0;

    // device copies of the initialised arrays
    int32_t *d_blocks = nullptr;
    int64_t *d_blk_off = nullptr;
    int32_t *d_I_V = nullptr, *d_I_T = nullptr;
    int64_t *d_sizes = nullptr;  // [(K+NP)*5] clusters, then parts
    gale::PartInfo *d_parts = nullptr;  // [NP]
    int32_t *d_tt_pos = nullptr;        // [nt] TT row offsets of the cut clusters' internal tets
    int32_t *d_tt_general = nullptr;    // [K] counting pass: 1 where a cluster's TT takes the general pass
    int32_t *d_all_items = nullptr;     // [n_all] the full build's item list (cut clusters replaced by their parts)
    std::vector<int32_t> all_items;     // host copy
    std::vector<int32_t> pos_all;       // [K+NP] position of each item in all_items (-1: a cut cluster)
    int32_t *d_err = nullptr;
    int32_t last_err_word = 0;          // the device error word check_device_error last read
    int32_t *d_tickets = nullptr;  // one per bin (+ spare)
    int32_t *d_ids = nullptr;      // [K+NP] item ids of a partial build
    int32_t *d_order_all = nullptr;   // [K+NP] per bin: positions in all_items (largest first)
    int32_t *d_order_ids = nullptr;   // [K+NP] per bin: item ids (the counting pass)
    int32_t *d_order_part = nullptr;  // [K+NP] order of a partial build
    gale::WorkItem *d_items = nullptr;      // [K+NP]
    gale::WorkItem *d_arrays_base = nullptr;  // [16] base pointers per mask
    int64_t *d_totals = nullptr;            // [10]
    int64_t *d_bsum = nullptr;              // output placement scratch
    char *d_spill = nullptr;                // per-CTA regions of spill bins
    gale::SmemPlan *d_plans = nullptr;      // [K+NP] own plans of the members of per-item bins
    std::vector<gale::SmemPlan> h_plans;    // host copy
    int64_t spill_bytes = 0;
    std::vector<int64_t> sizes;             // host [(K+NP)*5]
    std::vector<int32_t> tt_general;        // host [K]: 1 where the cluster is non-manifold (TT general pass)
    int64_t totals[5] = {0, 0, 0, 0, 0};
    double device_seconds = 0;

    // size bins
    std::vector<gale::Bin> bins;
    std::vector<int32_t> bin_of;        // [K+NP]
    std::vector<int64_t> order_all_off; // [nbins+1] offsets into d_order_all
    int threads_override = 0;  // 0: chosen from the cluster's tet count
    int ctas_override = 0;
    int sm_count = 0;

    // bulk output arrays
    int32_t *bulk[10] = {};
    int64_t bulk_cap[10] = {};
    int64_t bulk_len[10] = {};
    std::vector<int64_t> bulk_offs;  // [n*10]
    std::vector<int32_t> bulk_ids;
    uint32_t bulk_mask = 0;

    // pipelined build + export: copy stream, chunk events, chunk base items
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> chunk_events;
    gale::WorkItem *d_chunk_base = nullptr;  // [kMaxExportChunks]

    // device -> host copies into pageable memory (gale::copy_to_host): two
    // pinned staging buffers, allocated on first use
    void *stage[2] = {};
    cudaEvent_t stage_ev[2] = {};
    std::mutex stage_mu;

    // captured full builds, one per mask
    cudaGraphExec_t graphs[16] = {};
    int64_t last_launches = 0;

    std::vector<gale::DevAlloc> allocs;
    std::mutex mu;  // guards builds and the bulk state

    gale::Serve *serve = nullptr;
    gale::Enumeration *enm = nullptr;  // built by gale_enumerate
    gale::Cobound *cb = nullptr;       // gale_build_coboundary
    int32_t serve_mode = -1;          // -1: default (loop when it fits)
    int64_t serve_idle_us = 0;
    int32_t serve_loop_ctas = 0;      // 0: as many as fit
    int32_t serve_prefetch = 0;       // clusters queued ahead of each request
    int64_t serve_lease_ns = 0;       // 0: pins never expire

    void *dalloc(size_t bytes);
    void dfree(void *p);
};

namespace gale {
// Synchronous device -> host copy of `bytes` on the context stream: one copy
// into page-locked memory; into pageable memory through the staging buffers,
// moved into place by the host threads (gale_api.cpp).
gale_status copy_to_host(gale_ctx *ctx, void *dst, const void *src, size_t bytes);
// Lengths of the ten output arrays of cluster k under mask (gale_api.cpp).
void item_lengths(const gale_ctx *ctx, int32_t k, uint32_t mask, int64_t *L);
void enumeration_destroy(gale_ctx *ctx);  // gale_enum.cpp
void cobound_destroy(gale_ctx *ctx);      // gale_cobound.cu
}  // namespace gale
