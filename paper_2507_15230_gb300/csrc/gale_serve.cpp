// Serving: consumer requests for whole clusters (Section 4.4), admitted
// against an HBM budget, built on the device and kept in an LRU relation
// cache (Section 4.5's leader producer, re-designed).
//
// A consumer thread calls gale_request(cluster, mask).  A cached entry whose
// mask covers the request is a hit: it is pinned and returned at once.  A
// miss creates an entry and queues it for the leader thread, which
//   - admits queued entries in arrival order against the budget: each gets a
//     slot in one device slab (first fit, coalescing free list), evicting
//     unpinned ready entries least-recently-used first; prefetched clusters
//     (Section 4.5's proactive computation) wait in a queue of their own and
//     are admitted only while no request waits, with at most half the loop's
//     CTAs busy on them, into free space only (a prefetch never evicts, and
//     is dropped when the budget is full), and a request for a cluster still
//     queued as a prefetch moves it to the request queue;
//   - writes each admitted entry's work item (its cluster, mask and output
//     pointers into its slot) into a ring in pinned, mapped host memory and
//     publishes its ticket (release store of the ring tail);
//   - keeps the device-resident loop running: persistent CTAs claim
//     published tickets, build, and store the ticket into the slot's done
//     flag; the loop exits after an idle period and is relaunched when
//     published work is pending;
//   - polls the done flags, marks entries ready and wakes the waiters.
// Requests that arrive while others are on the device are admitted as slots
// and memory free up and are picked up by the running loop without a new
// launch (continuous batching).  When the merged shared-memory plan of all
// size bins does not fit one CTA, the leader instead launches the persistent
// build kernel per bin for each batch of admitted entries and completes them
// through a CUDA event (launch mode).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <set>
#include <memory>
#include <thread>
#include <unordered_map>

#ifdef __linux__
#include <sys/prctl.h>
#endif

#include "gale_ctx.h"

namespace gale {

// defined in gale_api.cpp
SmemPlan serve_plan(gale_ctx *ctx, bool *fits, std::vector<uint8_t> *in_loop, std::vector<SmemPlan> *own = nullptr);

namespace {

constexpr int32_t kRingCap = 4096;
constexpr int64_t kAlign = 256;

inline int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

enum class St { Queued, Building, Ready, Failed };

struct Entry {
    int32_t k;
    uint32_t mask;
    St state = St::Queued;
    int32_t refs = 0;
    int64_t off = -1, bytes = 0;  // slot in the slab
    int64_t ticket = -1;
    gale_status fail = GALE_OK;
    WorkItem item{};
    int64_t n_edges = 0;
    std::list<Entry *>::iterator lru;  // valid when Ready and unpinned-or-pinned (always in lru when Ready)
    bool in_lru = false;
    bool prefetch = false;  // queued ahead of any request
    bool claimed = false;   // a request has used it
    int64_t t_queued = 0, t_admitted = 0, t_published = 0;  // steady-clock ns of each stage
    std::condition_variable cv;  // its waiters: woken when it becomes ready or fails
};

// one view handed out by gale_request
struct Pin {
    Entry *e;
    int64_t deadline;  // steady-clock ns; INT64_MAX without a lease
};

// best-fit allocator over [0, cap): free blocks by offset (to coalesce a
// released block with its neighbours) and by size (to find the smallest
// block that fits, and whether any does, in logarithmic time)
struct Slab {
    std::map<int64_t, int64_t> free;             // offset -> size
    std::set<std::pair<int64_t, int64_t>> by_size;  // (size, offset)
    int64_t cap = 0, used = 0;
    void init(int64_t c) {
        cap = c;
        free.clear();
        by_size.clear();
        if (c > 0) add(0, c);
        used = 0;
    }
    void add(int64_t off, int64_t n) {
        free[off] = n;
        by_size.insert({n, off});
    }
    void drop(std::map<int64_t, int64_t>::iterator it) {
        by_size.erase({it->second, it->first});
        free.erase(it);
    }
    bool fits(int64_t n) const { return !by_size.empty() && by_size.rbegin()->first >= n; }
    int64_t alloc(int64_t n) {
        auto b = by_size.lower_bound({n, INT64_MIN});
        if (b == by_size.end()) return -1;
        const int64_t sz = b->first, off = b->second;
        drop(free.find(off));
        if (sz > n) add(off + n, sz - n);
        used += n;
        return off;
    }
    void release(int64_t off, int64_t n) {
        used -= n;
        auto nx = free.lower_bound(off);
        if (nx != free.end() && off + n == nx->first) {
            n += nx->second;
            auto del = nx++;
            drop(del);
        }
        if (nx != free.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                off = pv->first;
                n += pv->second;
                drop(pv);
            }
        }
        add(off, n);
    }
};

}  // namespace

struct Serve {
    gale_ctx *ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv_leader; // work for the leader
    std::unordered_map<int64_t, std::unique_ptr<Entry>> entries;  // key = k * 16 + mask
    std::deque<Entry *> queue;           // requested entries waiting for admission, in arrival order
    std::deque<Entry *> pqueue;          // prefetch entries waiting for admission
    int64_t inflight_prefetch = 0;       // prefetch entries on the device
    std::list<Entry *> lru;              // ready entries, most recent first
    Slab slab;
    char *slab_base = nullptr;
    bool stop = false;
    std::thread leader;
    gale_serve_stats stats{};
    std::unordered_map<uint64_t, Pin> pins;  // handle -> pinned entry
    uint64_t next_pin = 1;
    int64_t lease_ns = 0;
    int64_t next_lease_scan = 0;

    // device loop (clusters of the bins it covers; the others are batched)
    bool loop_mode = true;
    std::vector<uint8_t> in_loop;  // per size bin
    bool single_mode = false;  // one launch per request (baseline form)
    SmemPlan plan{};               // launch envelope of the loop
    SmemPlan *d_plans = nullptr;   // [K] the plan each cluster the loop serves is built under
    int grid = 0;
    WorkItem *h_items = nullptr;   // mapped
    long long *h_tail = nullptr;   // mapped
    long long *h_done = nullptr;   // mapped [cap]
    long long *h_times = nullptr;  // mapped [2 cap]: device clock at claim and completion
    int *h_stop = nullptr;         // mapped
    WorkItem *d_items = nullptr;
    long long *d_tail = nullptr, *d_done = nullptr, *d_times = nullptr;
    int *d_stop = nullptr;
    unsigned long long *d_next = nullptr;
    int32_t *d_err = nullptr;
    cudaStream_t loop_stream = nullptr;
    cudaEvent_t loop_event = nullptr;
    bool loop_launched = false;
    bool loop_seen_running = false;  // this leader iteration found the loop still running
    int64_t last_leader_ns = 0;      // end of the leader thread's last step of the state machine
    long long published = 0;      // tickets published
    std::map<long long, Entry *> inflight;  // ticket -> entry
    uint64_t idle_ns = 20ull * 1000 * 1000;

    // launch mode
    WorkItem *d_batch = nullptr;   // [kRingCap] device work items
    int32_t *d_border = nullptr;   // [kRingCap] per-bin order
    int32_t *d_tick = nullptr;     // [kMaxBins] tickets
    WorkItem *h_batch = nullptr;   // pinned staging
    int32_t *h_border = nullptr;
    cudaEvent_t batch_event = nullptr;
    cudaStream_t batch_stream = nullptr;  // batched launches, beside the loop
    char *d_spill = nullptr;       // large-cluster scratch of the serving stream
    std::vector<Entry *> batch_entries;
    bool batch_busy = false;

    gale_status init(gale_ctx *c);
    void leader_loop();
    bool pump(bool poll = true);
    bool admit(Entry *e);
    void fill_item(Entry *e);
    void publish_loop(Entry *e);
    void poll_loop();
    void launch_batch(std::vector<Entry *> &b);
    void poll_batch();
    void evict_for(int64_t bytes);
    bool expire_leases();
    void stage_done(Entry *e);
    int64_t entry_bytes(int32_t k, uint32_t mask, int64_t *L);
};

namespace {

gale_status fail(gale_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

inline int64_t a256(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace

int64_t Serve::entry_bytes(int32_t k, uint32_t mask, int64_t *L) {
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
    int64_t b = 0;
    for (int a = 0; a < 10; ++a) b += (L[a] * 4 + 15) / 16 * 16;
    return a256(b);
}

gale_status Serve::init(gale_ctx *c) {
    ctx = c;
    stats.cache_bytes_budget = ctx->cache_budget;
    slab_base = static_cast<char *>(ctx->dalloc(size_t(ctx->cache_budget)));
    if (!slab_base) return fail(GALE_ENOMEM, "device allocation of the relation cache failed");
    slab.init(ctx->cache_budget);
    bool fits = false;
    std::vector<SmemPlan> own;
    plan = serve_plan(ctx, &fits, &in_loop, &own);
    loop_mode = fits && (ctx->serve_mode < 0 || ctx->serve_mode == GALE_SERVE_LOOP);
    single_mode = ctx->serve_mode == GALE_SERVE_SINGLE;
    if (ctx->serve_idle_us > 0) idle_ns = uint64_t(std::max<int64_t>(100, ctx->serve_idle_us)) * 1000ull;
    lease_ns = ctx->serve_lease_ns;
    auto ck = [](cudaError_t e) { return e == cudaSuccess; };
    if (!ck(cudaHostAlloc(reinterpret_cast<void **>(&h_items), sizeof(WorkItem) * kRingCap, cudaHostAllocMapped)) ||
        !ck(cudaHostAlloc(reinterpret_cast<void **>(&h_tail), 64, cudaHostAllocMapped)) ||
        !ck(cudaHostAlloc(reinterpret_cast<void **>(&h_done), sizeof(long long) * kRingCap, cudaHostAllocMapped)) ||
        !ck(cudaHostAlloc(reinterpret_cast<void **>(&h_stop), 64, cudaHostAllocMapped)) ||
        !ck(cudaHostAlloc(reinterpret_cast<void **>(&h_times), sizeof(long long) * 2 * kRingCap,
                          cudaHostAllocMapped)) ||
        !ck(cudaHostAlloc(reinterpret_cast<void **>(&h_batch), sizeof(WorkItem) * kRingCap, cudaHostAllocDefault)) ||
        !ck(cudaHostAlloc(reinterpret_cast<void **>(&h_border), sizeof(int32_t) * kRingCap, cudaHostAllocDefault)))
        return fail(GALE_ENOMEM, "pinned host allocation for the serving ring failed");
    *h_tail = 0;
    *h_stop = 0;
    for (int i = 0; i < kRingCap; ++i) h_done[i] = -1;
    if (!ck(cudaHostGetDevicePointer(reinterpret_cast<void **>(&d_items), h_items, 0)) ||
        !ck(cudaHostGetDevicePointer(reinterpret_cast<void **>(&d_tail), h_tail, 0)) ||
        !ck(cudaHostGetDevicePointer(reinterpret_cast<void **>(&d_done), h_done, 0)) ||
        !ck(cudaHostGetDevicePointer(reinterpret_cast<void **>(&d_stop), h_stop, 0)) ||
        !ck(cudaHostGetDevicePointer(reinterpret_cast<void **>(&d_times), h_times, 0)))
        return fail(GALE_ECUDA, "mapping the serving ring failed");
    d_plans = static_cast<SmemPlan *>(ctx->dalloc(sizeof(SmemPlan) * size_t(std::max(ctx->hm.K, 1))));
    if (!d_plans) return fail(GALE_ENOMEM, "device allocation of the serving plans failed");
    if (ctx->hm.K > 0 &&
        cudaMemcpy(d_plans, own.data(), sizeof(SmemPlan) * size_t(ctx->hm.K), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(GALE_ECUDA, "uploading the serving plans failed");
    d_next = static_cast<unsigned long long *>(ctx->dalloc(64));
    d_err = static_cast<int32_t *>(ctx->dalloc(64));
    d_batch = static_cast<WorkItem *>(ctx->dalloc(sizeof(WorkItem) * kRingCap));
    d_border = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * kRingCap));
    d_tick = static_cast<int32_t *>(ctx->dalloc(sizeof(int32_t) * kMaxBins));
    if (!d_next || !d_err || !d_batch || !d_border || !d_tick)
        return fail(GALE_ENOMEM, "device allocation for the serving loop failed");
    if (ctx->spill_bytes > 0) {
        d_spill = static_cast<char *>(ctx->dalloc(size_t(ctx->spill_bytes)));
        if (!d_spill) return fail(GALE_ENOMEM, "device allocation of the serving large-cluster scratch failed");
    }
    if (!ck(cudaStreamCreateWithFlags(&loop_stream, cudaStreamNonBlocking)) ||
        !ck(cudaStreamCreateWithFlags(&batch_stream, cudaStreamNonBlocking)) ||
        !ck(cudaEventCreateWithFlags(&loop_event, cudaEventDisableTiming)) ||
        !ck(cudaEventCreateWithFlags(&batch_event, cudaEventDisableTiming)) ||
        !ck(cudaMemsetAsync(d_next, 0, 64, loop_stream)) || !ck(cudaMemsetAsync(d_err, 0, 64, loop_stream)) ||
        !ck(cudaStreamSynchronize(loop_stream)))
        return fail(GALE_ECUDA, "creating the serving stream failed");
    if (loop_mode) {
        const int per_sm = serve_ctas_per_sm(plan);
        if (per_sm < 1) loop_mode = false;
        else grid = per_sm * ctx->sm_count;
        if (ctx->serve_loop_ctas > 0) grid = std::min(grid, ctx->serve_loop_ctas);
    }
    try {
        leader = std::thread([this] { leader_loop(); });
    } catch (const std::exception &) {
        return fail(GALE_ENOMEM, "the serving leader thread could not be started");
    }
    return GALE_OK;
}

void Serve::evict_for(int64_t bytes) {
    // evict unpinned ready entries, least recently used first, until a free
    // block of `bytes` exists or nothing more can go
    for (;;) {
        if (slab.fits(bytes)) return;
        auto victim = lru.end();
        for (auto it = lru.end(); it != lru.begin();) {
            --it;
            if ((*it)->refs == 0) {
                victim = it;
                break;
            }
        }
        if (victim == lru.end()) return;
        Entry *e = *victim;
        lru.erase(victim);
        e->in_lru = false;
        slab.release(e->off, e->bytes);
        stats.evictions++;
        entries.erase(int64_t(e->k) * 16 + e->mask);  // frees e
    }
}

bool Serve::admit(Entry *e) {
    int64_t L[10];
    const int64_t bytes = entry_bytes(e->k, e->mask, L);
    if (bytes > slab.cap) {
        e->state = St::Failed;
        e->fail = GALE_ENOMEM;
        e->cv.notify_all();
        return true;
    }
    int64_t off = slab.alloc(bytes);
    if (off < 0 && !e->prefetch) {  // a prefetch takes free space only: it never evicts
        evict_for(bytes);
        off = slab.alloc(bytes);
    }
    if (off < 0) return false;  // budget full (or pinned): wait for releases, or drop a prefetch
    e->off = off;
    e->bytes = bytes;
    fill_item(e);
    e->t_admitted = now_ns();
    if (!e->prefetch) {
        const int64_t w = e->t_admitted - e->t_queued;
        stats.t_queue_ns += w;
        stats.max_queue_ns = std::max(stats.max_queue_ns, w);
        int b = 0;
        while (b < 15 && (int64_t(2000) << b) <= w) ++b;
        stats.queue_hist[b]++;
    }
    return true;
}

// an entry's build finished: it joins the LRU list
void Serve::stage_done(Entry *e) {
    if (e->prefetch) inflight_prefetch--;
    e->state = St::Ready;
    lru.push_front(e);
    e->lru = lru.begin();
    e->in_lru = true;
    stats.builds++;
    e->cv.notify_all();
    if (!e->prefetch) stats.t_build_ns += now_ns() - e->t_published;
}

// revoke the pins whose lease ran out; true if any was
bool Serve::expire_leases() {
    if (lease_ns <= 0 || pins.empty()) return false;
    const int64_t now = now_ns();
    if (now < next_lease_scan) return false;
    next_lease_scan = now + std::min<int64_t>(lease_ns / 4 + 1, 1000000);
    bool any = false;
    for (auto it = pins.begin(); it != pins.end();) {
        if (it->second.deadline <= now) {
            it->second.e->refs--;
            stats.leases_expired++;
            it = pins.erase(it);
            any = true;
        } else {
            ++it;
        }
    }
    return any;
}

void Serve::fill_item(Entry *e) {
    int64_t L[10];
    entry_bytes(e->k, e->mask, L);
    int32_t *p[10];
    char *cur = slab_base + e->off;
    for (int a = 0; a < 10; ++a) {
        p[a] = reinterpret_cast<int32_t *>(cur);
        cur += (L[a] * 4 + 15) / 16 * 16;
    }
    const uint32_t m = e->mask;
    WorkItem &w = e->item;
    w.k = e->k;
    w.mask = m;
    w.blk = ctx->hm.blk_off[e->k];
    w.vt_off = (m & GALE_VT) ? p[0] : nullptr;
    w.vt_val = (m & GALE_VT) ? p[1] : nullptr;
    w.vv_off = (m & GALE_VV) ? p[2] : nullptr;
    w.vv_val = (m & GALE_VV) ? p[3] : nullptr;
    w.eu_off = (m & GALE_ET) ? p[4] : nullptr;
    w.e_w = (m & GALE_ET) ? p[5] : nullptr;
    w.et_off = (m & GALE_ET) ? p[6] : nullptr;
    w.et_val = (m & GALE_ET) ? p[7] : nullptr;
    w.tt_off = (m & GALE_TT) ? p[8] : nullptr;
    w.tt_val = (m & GALE_TT) ? p[9] : nullptr;
    e->n_edges = ctx->sizes[size_t(5) * e->k + 2];
}

void Serve::publish_loop(Entry *e) {
    const long long t = published;
    const int slot = int(t % kRingCap);
    h_items[slot] = e->item;
    __atomic_store_n(h_tail, t + 1, __ATOMIC_RELEASE);
    published = t + 1;
    e->ticket = t;
    e->state = St::Building;
    if (e->prefetch) inflight_prefetch++;
    e->t_published = now_ns();
    if (!e->prefetch) stats.t_prepare_ns += e->t_published - e->t_admitted;
    inflight[t] = e;
    // one event query per leader iteration: a running loop claims every
    // ticket published while it runs
    if (!loop_launched || (!loop_seen_running && cudaEventQuery(loop_event) == cudaSuccess)) {
        // (re)start the loop; a previous one has drained or never ran
        const DevMesh dm{ctx->d_blocks, ctx->d_blk_off, ctx->d_I_V, ctx->d_I_T, ctx->hm.K};
        ServeRing ring{d_items, d_tail, d_done, d_stop, d_next, kRingCap, 0, idle_ns, d_times};
        launch_serve(dm, plan, d_plans, ring, d_err, grid, loop_stream);
        cudaEventRecord(loop_event, loop_stream);
        loop_launched = true;
        stats.batches++;
    }
    loop_seen_running = true;
}

void Serve::poll_loop() {
    for (auto it = inflight.begin(); it != inflight.end();) {
        const long long t = it->first;
        if (__atomic_load_n(h_done + (t % kRingCap), __ATOMIC_ACQUIRE) == t) {
            Entry *e = it->second;
            if (!e->prefetch) {
                const int slot = int(t % kRingCap);
                stats.t_kernel_ns += h_times[2 * slot + 1] - h_times[2 * slot];
            }
            stage_done(e);
            it = inflight.erase(it);
        } else {
            ++it;
        }
    }
    // published work with no loop running (it drained just before): restart
    if (!inflight.empty() && loop_launched && cudaEventQuery(loop_event) == cudaSuccess) {
        const DevMesh dm{ctx->d_blocks, ctx->d_blk_off, ctx->d_I_V, ctx->d_I_T, ctx->hm.K};
        ServeRing ring{d_items, d_tail, d_done, d_stop, d_next, kRingCap, 0, idle_ns, d_times};
        launch_serve(dm, plan, d_plans, ring, d_err, grid, loop_stream);
        cudaEventRecord(loop_event, loop_stream);
        stats.batches++;
    }
}

void Serve::launch_batch(std::vector<Entry *> &b) {
    // per-bin order over the batch, largest working sets first
    const int nb = int(ctx->bins.size());
    std::vector<std::vector<int32_t>> per(nb);
    for (int32_t i = 0; i < int32_t(b.size()); ++i) {
        h_batch[i] = b[i]->item;
        per[ctx->bin_of[b[i]->k]].push_back(i);
    }
    int32_t n = 0;
    std::vector<int32_t> off(nb + 1, 0);
    for (int bb = 0; bb < nb; ++bb) {
        for (int32_t i : per[bb]) h_border[n++] = i;
        off[bb + 1] = n;
    }
    cudaMemcpyAsync(d_batch, h_batch, sizeof(WorkItem) * b.size(), cudaMemcpyHostToDevice, batch_stream);
    cudaMemcpyAsync(d_border, h_border, sizeof(int32_t) * n, cudaMemcpyHostToDevice, batch_stream);
    const DevMesh dm{ctx->d_blocks, ctx->d_blk_off, ctx->d_I_V, ctx->d_I_T, ctx->hm.K};
    int rc = 0;
    for (int bb = 0; bb < nb && rc == 0; ++bb) {
        const int32_t m = off[bb + 1] - off[bb];
        if (m == 0) continue;
        char *scr = ctx->bins[bb].spill ? d_spill : nullptr;
        if (single_mode)
            rc = launch_build_one(dm, ctx->bins[bb].per_item ? ctx->h_plans[b[h_border[off[bb]]]->k] : ctx->bins[bb].plan,
                                  d_batch, h_border[off[bb]], d_err, batch_stream, scr);
        else
            rc = launch_build(dm, ctx->bins[bb].plan, d_batch, d_border + off[bb], m, d_err, d_tick + bb,
                              std::min(ctx->bins[bb].grid, m), batch_stream, scr,
                              ctx->bins[bb].per_item ? ctx->d_plans : nullptr);
    }
    if (rc != 0) {
        // nothing of this batch is trusted: its entries fail and free their space
        for (Entry *e : b) {
            e->state = St::Failed;
            e->fail = GALE_ECUDA;
            e->cv.notify_all();
            slab.release(e->off, e->bytes);
            e->bytes = 0;
            if (e->prefetch && e->refs == 0) entries.erase(int64_t(e->k) * 16 + e->mask);  // frees e
        }
        cudaStreamSynchronize(batch_stream);
        return;
    }
    cudaEventRecord(batch_event, batch_stream);
    const int64_t tp = now_ns();
    for (Entry *e : b) {
        e->state = St::Building;
        e->t_published = tp;
        if (e->prefetch) inflight_prefetch++;
        if (!e->prefetch) stats.t_prepare_ns += tp - e->t_admitted;
    }
    batch_entries = b;
    batch_busy = true;
    stats.batches++;
}

void Serve::poll_batch() {
    if (!batch_busy || cudaEventQuery(batch_event) != cudaSuccess) return;
    for (Entry *e : batch_entries) stage_done(e);
    batch_entries.clear();
    batch_busy = false;
}

// One step of the serving state machine, with mu held: admission (requested
// entries in arrival order, then prefetches while no request waits and few
// prefetches occupy the device, so that a request never queues behind work
// nobody has asked for yet), publication or batched launches, and polling of
// the device for finished entries (unless poll is false).  The leader thread
// runs it in a loop, and so does every requesting thread while it waits: a
// request's progress never depends on the leader thread getting a core
// (consumer threads that compute between requests can fill every core of the
// host).  Returns true while work is queued or on the device.
bool Serve::pump(bool poll) {
    int dev_before = -1;
    cudaGetDevice(&dev_before);
    if (dev_before != ctx->device) cudaSetDevice(ctx->device);
    loop_seen_running = false;
    bool progressed = expire_leases();
    std::vector<Entry *> batch;
    const int64_t prefetch_cap = loop_mode ? std::max(1, grid / 2) : kRingCap / 2;
    for (int pass = 0; pass < 2; ++pass) {
        std::deque<Entry *> &q = pass == 0 ? queue : pqueue;
        if (pass == 1 && !queue.empty()) break;
        while (!q.empty()) {
            Entry *e = q.front();
            if (pass == 1 && inflight_prefetch + int64_t(batch.size()) >= prefetch_cap) break;
            const bool via_loop = loop_mode && in_loop[ctx->bin_of[e->k]];
            if (!via_loop && batch_busy) break;
            if (via_loop && published - (inflight.empty() ? published : inflight.begin()->first) >= kRingCap) break;
            if (!admit(e)) {
                if (!(e->prefetch && e->refs == 0)) break;
                // a prefetch waits for nothing: drop it while the budget is full
                q.pop_front();
                stats.prefetch_dropped++;
                entries.erase(int64_t(e->k) * 16 + e->mask);  // frees e
                progressed = true;
                continue;
            }
            q.pop_front();
            progressed = true;
            if (e->state == St::Failed) {
                if (e->prefetch && e->refs == 0) entries.erase(int64_t(e->k) * 16 + e->mask);
                continue;
            }
            if (via_loop) publish_loop(e);
            else {
                batch.push_back(e);
                if (int(batch.size()) >= (single_mode ? 1 : kRingCap)) break;
            }
        }
        if (int(batch.size()) >= (single_mode ? 1 : kRingCap)) break;
    }
    if (!batch.empty()) launch_batch(batch);
    const size_t before = inflight.size() + (batch_busy ? batch_entries.size() : 0);
    if (poll) {
        if (loop_mode) poll_loop();
        poll_batch();
    }
    const size_t after = inflight.size() + (batch_busy ? batch_entries.size() : 0);
    if (after != before || progressed) stats.max_batch = std::max<int64_t>(stats.max_batch, int64_t(before));
    if (const size_t pending = queue.size() + pqueue.size() + after) {
        int b = 0;
        while (b < 11 && (size_t(2) << b) <= pending) ++b;
        stats.depth_hist[b]++;
    }
    stats.cache_bytes_used = slab.used;
    stats.max_prefetch_queue = std::max<int64_t>(stats.max_prefetch_queue, int64_t(pqueue.size()));
    if (dev_before >= 0 && dev_before != ctx->device) cudaSetDevice(dev_before);
    return after > 0 || !queue.empty() || !pqueue.empty();
}

void Serve::leader_loop() {
    cudaSetDevice(ctx->device);
#ifdef __linux__
    // the leader sleeps a few us between polls while work is in flight (with
    // the lock released, so requests queue meanwhile); the default 50 us
    // timer slack would stretch every such sleep to ~60 us
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        const int64_t pass_t0 = now_ns();
        const bool busy = pump();
        last_leader_ns = now_ns();
        const int64_t hold = last_leader_ns - pass_t0;
        stats.leader_passes++;
        stats.leader_hold_ns += hold;
        stats.max_leader_hold_ns = std::max(stats.max_leader_hold_ns, hold);
        if (busy) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(2));
            lk.lock();
        } else {
            cv_leader.wait_for(lk, std::chrono::milliseconds(50));
        }
    }
}

void serve_destroy(gale_ctx *ctx) {
    Serve *s = ctx->serve;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_leader.notify_all();
    if (s->leader.joinable()) s->leader.join();
    if (s->h_stop) __atomic_store_n(s->h_stop, 1, __ATOMIC_RELEASE);
    if (s->loop_stream) cudaStreamSynchronize(s->loop_stream);
    if (s->batch_stream) cudaStreamSynchronize(s->batch_stream);
    if (s->loop_event) cudaEventDestroy(s->loop_event);
    if (s->batch_event) cudaEventDestroy(s->batch_event);
    if (s->loop_stream) cudaStreamDestroy(s->loop_stream);
    if (s->batch_stream) cudaStreamDestroy(s->batch_stream);
    cudaFreeHost(s->h_items);
    cudaFreeHost(s->h_tail);
    cudaFreeHost(s->h_done);
    cudaFreeHost(s->h_stop);
    cudaFreeHost(s->h_times);
    cudaFreeHost(s->h_batch);
    cudaFreeHost(s->h_border);
    delete s;
    ctx->serve = nullptr;
}

}  // namespace gale

using gale::Entry;
using gale::St;

namespace {

gale_status fail(gale_status s, const std::string &msg) {
    gale::set_error(msg);
    return s;
}

std::mutex g_serve_init_mu;

gale_status ensure_serve(gale_ctx *ctx) {
    std::lock_guard<std::mutex> lk(g_serve_init_mu);
    if (ctx->serve) return GALE_OK;
    if (ctx->cache_budget <= 0) return fail(GALE_EINVAL, "serving needs cache_budget_bytes > 0 at load");
    auto *s = new gale::Serve();
    ctx->serve = s;
    gale_status st = s->init(ctx);
    if (st != GALE_OK) {
        std::string keep = gale_last_error();
        gale::serve_destroy(ctx);
        return fail(st, keep);
    }
    return GALE_OK;
}

void fill_view(gale_ctx *ctx, Entry *e, gale_view *out) {
    memset(out, 0, sizeof(*out));
    const int32_t k = e->k;
    out->cluster = k;
    out->mask = e->mask;
    out->v_begin = ctx->hm.I_V[k];
    out->v_end = ctx->hm.I_V[k + 1];
    out->t_begin = ctx->hm.I_T[k];
    out->t_end = ctx->hm.I_T[k + 1];
    out->n_edges = int32_t(e->n_edges);
    const gale::WorkItem &w = e->item;
    out->vt_off = w.vt_off;
    out->vt_val = w.vt_val;
    out->vv_off = w.vv_off;
    out->vv_val = w.vv_val;
    out->et_uoff = w.eu_off;
    out->et_w = w.e_w;
    out->et_off = w.et_off;
    out->et_val = w.et_val;
    out->tt_off = w.tt_off;
    out->tt_val = w.tt_val;
}

// hand out a pin of e (whose refs the caller has already counted)
void issue(gale_ctx *ctx, gale::Serve *s, Entry *e, gale_view *out, int64_t t0) {
    fill_view(ctx, e, out);
    const uint64_t id = s->next_pin++;
    const int64_t now = gale::now_ns();
    s->pins[id] = gale::Pin{e, s->lease_ns > 0 ? now + s->lease_ns : INT64_MAX};
    out->handle = id;
    s->stats.t_wait_ns += now - t0;
    s->stats.max_wait_ns = std::max<int64_t>(s->stats.max_wait_ns, now - t0);
}

}  // namespace

extern "C" {

gale_status gale_request(gale_ctx *ctx, int32_t cluster_id, uint32_t mask, int64_t timeout_ns, gale_view *out) {
    if (!ctx || !out) return fail(GALE_EINVAL, "NULL argument");
    if (ctx->device < 0) return fail(GALE_EINVAL, "host-only context");
    if (cluster_id < 0 || cluster_id >= ctx->hm.K) return fail(GALE_EINVAL, "cluster id out of range");
    if (mask == 0 || (mask & ~ctx->precond))
        return fail(GALE_EINVAL, "mask must be a non-empty subset of the precondition mask");
    gale_status st = ensure_serve(ctx);
    if (st != GALE_OK) return st;
    gale::Serve *s = ctx->serve;
    const int64_t t0 = gale::now_ns();
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns > 0 ? timeout_ns : 0);
    std::unique_lock<std::mutex> lk(s->mu);
    s->stats.requests++;
    Entry *e = nullptr;
    // a cached entry whose mask covers the request
    for (uint32_t m = 1; m < 16 && !e; ++m) {
        if ((m & mask) != mask) continue;
        auto it = s->entries.find(int64_t(cluster_id) * 16 + m);
        if (it != s->entries.end() && it->second->state != St::Failed) e = it->second.get();
    }
    if (e && e->prefetch && !e->claimed) {
        e->claimed = true;
        s->stats.prefetch_hits++;
        if (e->state == St::Queued) {
            // still waiting as a prefetch: it becomes a request, queued now
            auto pit = std::find(s->pqueue.begin(), s->pqueue.end(), e);
            if (pit != s->pqueue.end()) s->pqueue.erase(pit);
            e->prefetch = false;
            e->t_queued = gale::now_ns();
            s->stats.promotions++;
            s->queue.push_back(e);
            s->cv_leader.notify_all();
        }
    }
    if (e && e->state == St::Ready) {
        s->stats.hits++;
        e->refs++;
        s->lru.splice(s->lru.begin(), s->lru, e->lru);
        s->stats.t_enqueue_ns += gale::now_ns() - t0;
        issue(ctx, s, e, out, t0);
        return GALE_OK;
    }
    if (!e) {
        s->stats.misses++;
        auto ne = std::make_unique<Entry>();
        ne->k = cluster_id;
        ne->mask = mask;
        e = ne.get();
        e->t_queued = gale::now_ns();
        s->entries[int64_t(cluster_id) * 16 + mask] = std::move(ne);
        s->queue.push_back(e);
        s->cv_leader.notify_all();
    }
    s->stats.t_enqueue_ns += gale::now_ns() - t0;
    // proactive prefetch: the following clusters, queued behind the request
    for (int32_t j = 1; j <= ctx->serve_prefetch && cluster_id + j < ctx->hm.K; ++j) {
        const int32_t kk = cluster_id + j;
        bool have = false;
        for (uint32_t m = 1; m < 16 && !have; ++m) {
            if ((m & mask) != mask) continue;
            auto it = s->entries.find(int64_t(kk) * 16 + m);
            have = it != s->entries.end() && it->second->state != St::Failed;
        }
        if (have) continue;
        auto pe = std::make_unique<Entry>();
        pe->k = kk;
        pe->mask = mask;
        pe->prefetch = true;
        pe->t_queued = gale::now_ns();
        s->pqueue.push_back(pe.get());
        s->entries[int64_t(kk) * 16 + mask] = std::move(pe);
        s->stats.prefetches++;
    }
    e->refs++;
    auto ready = [&] { return e->state == St::Ready || e->state == St::Failed; };
    // between short waits (woken early when another thread completes the
    // entry), the waiting thread drives the serving state machine itself
    // whenever the leader thread has not done so lately, and right away the
    // first time (so that its own entry is admitted and published without a
    // hand-off):
    // consumer threads that compute between requests can fill every core
    //
    // While the entry builds in the device loop, the waiter watches its own
    // done flag (mapped host memory) without the lock, yielding the core,
    // and completes the entry itself as soon as the flag is set: timed
    // waits of a few microseconds last tens of microseconds under the
    // default timer slack, and the leader may not be running.
    constexpr int64_t kLeaderGapNs = 20000;
    constexpr int64_t kWatchNs = 64000;
    auto own_done = [&] {
        return e->state == St::Building && e->ticket >= 0 &&
               __atomic_load_n(s->h_done + (e->ticket % gale::kRingCap), __ATOMIC_ACQUIRE) == e->ticket;
    };
    for (bool first = true; !ready(); first = false) {
        if (first || own_done() || gale::now_ns() - s->last_leader_ns > kLeaderGapNs) {
            s->pump();
            s->stats.requester_pumps++;
        }
        if (ready()) break;
        if (timeout_ns > 0 && std::chrono::steady_clock::now() >= deadline) {
            e->refs--;
            s->stats.t_wait_ns += gale::now_ns() - t0;
            return fail(GALE_ETIMEOUT, "request timed out");
        }
        if (e->state == St::Building && e->ticket >= 0) {
            const long long tk = e->ticket;  // the entry stays: this thread holds a reference
            lk.unlock();
            const int64_t until = gale::now_ns() + kWatchNs;
            while (__atomic_load_n(s->h_done + (tk % gale::kRingCap), __ATOMIC_ACQUIRE) != tk && gale::now_ns() < until)
                std::this_thread::yield();
            lk.lock();
        } else {
            e->cv.wait_for(lk, std::chrono::microseconds(20));
        }
    }
    if (e->state == St::Failed) {
        const gale_status f = e->fail;
        e->refs--;
        if (e->refs == 0) s->entries.erase(int64_t(e->k) * 16 + e->mask);
        return fail(f, f == GALE_ENOMEM ? "cluster relations exceed the whole cache budget"
                                        : "launching the cluster's build failed");
    }
    issue(ctx, s, e, out, t0);
    return GALE_OK;
}

gale_status gale_release(gale_ctx *ctx, gale_view *view) {
    if (!ctx || !view) return fail(GALE_EINVAL, "NULL argument");
    if (!ctx->serve || view->handle == 0) return fail(GALE_ENOTFOUND, "not a serving view");
    gale::Serve *s = ctx->serve;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->pins.find(view->handle);
    if (it == s->pins.end()) return fail(GALE_ENOTFOUND, "view is not pinned (released, or its lease ran out)");
    it->second.e->refs--;
    s->pins.erase(it);
    view->handle = 0;
    s->cv_leader.notify_all();  // a pinned budget may have freed up
    return GALE_OK;
}

gale_status gale_serve_configure(gale_ctx *ctx, int32_t mode, int64_t idle_us, int32_t loop_ctas, int32_t prefetch) {
    if (!ctx) return fail(GALE_EINVAL, "NULL context");
    if (mode < GALE_SERVE_LOOP || mode > GALE_SERVE_SINGLE) return fail(GALE_EINVAL, "unknown serving mode");
    if (loop_ctas < 0) return fail(GALE_EINVAL, "loop_ctas must be >= 0");
    if (prefetch < 0) return fail(GALE_EINVAL, "prefetch must be >= 0");
    std::lock_guard<std::mutex> lk(g_serve_init_mu);
    if (ctx->serve) return fail(GALE_EBUSY, "serving already started on this context");
    if (mode == GALE_SERVE_LOOP && ctx->device >= 0) {
        bool fits = false;
        gale::serve_plan(ctx, &fits, nullptr);
        if (!fits) return fail(GALE_EINVAL, "the serving loop's merged plan does not fit one CTA");
    }
    ctx->serve_mode = mode;
    ctx->serve_idle_us = idle_us;
    ctx->serve_loop_ctas = loop_ctas;
    ctx->serve_prefetch = prefetch;
    return GALE_OK;
}

gale_status gale_serve_set_lease(gale_ctx *ctx, int64_t lease_ns) {
    if (!ctx) return fail(GALE_EINVAL, "NULL context");
    if (lease_ns < 0) return fail(GALE_EINVAL, "lease_ns must be >= 0");
    std::lock_guard<std::mutex> lk(g_serve_init_mu);
    ctx->serve_lease_ns = lease_ns;
    if (ctx->serve) {
        std::lock_guard<std::mutex> lk2(ctx->serve->mu);
        ctx->serve->lease_ns = lease_ns;
    }
    return GALE_OK;
}

gale_status gale_serve_stats_get(gale_ctx *ctx, gale_serve_stats *out) {
    if (!ctx || !out) return fail(GALE_EINVAL, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->cache_bytes_budget = ctx->cache_budget;
    if (!ctx->serve) return GALE_OK;
    std::lock_guard<std::mutex> lk(ctx->serve->mu);
    *out = ctx->serve->stats;
    out->cache_bytes_used = ctx->serve->slab.used;
    out->cache_bytes_budget = ctx->cache_budget;
    return GALE_OK;
}

}  // extern "C"
