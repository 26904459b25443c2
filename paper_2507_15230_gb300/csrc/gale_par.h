// Host thread-parallel loops shared by the host-side parts of the library
// (internal).
#pragma once

#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>
#include <new>
#include <thread>
#include <utility>
#include <vector>

namespace gale {

// fn(tid) for tid in [0, p) on p threads.  Ranks whose thread cannot be
// started (no resources) run on the calling thread afterwards, so no
// exception leaves a C-ABI call and every rank still runs exactly once.
template <class F>
void run_ranks(int p, F &&fn) {
    std::vector<std::thread> th;
    int started = 0;
    try {
        th.reserve(size_t(p));
        for (; started < p; ++started) th.emplace_back([&fn, started] { fn(started); });
    } catch (const std::exception &) {
    }
    for (int i = started; i < p; ++i) fn(i);
    for (auto &t : th) t.join();
}

// Static split of [0, n) into nthreads contiguous ranges: f(begin, end, tid).
template <class F>
void parallel_for(int64_t n, int nthreads, F &&f) {
    if (n <= 0) return;
    int p = nthreads;
    if (int64_t(p) > n) p = int(n);
    if (p <= 1) {
        f(int64_t(0), n, 0);
        return;
    }
    run_ranks(p, [&](int i) { f(n * i / p, n * (i + 1) / p, i); });
}

// Work-stealing loop over [0, n) in small grains (uneven per-item cost):
// f(i, tid).
template <class F>
void parallel_dynamic(int64_t n, int nthreads, int64_t grain, F &&f) {
    if (n <= 0) return;
    std::atomic<int64_t> next{0};
    int p = nthreads;
    if (int64_t(p) > (n + grain - 1) / grain) p = int((n + grain - 1) / grain);
    auto body = [&](int tid) {
        for (;;) {
            int64_t b = next.fetch_add(grain);
            if (b >= n) break;
            int64_t e = std::min(n, b + grain);
            for (int64_t i = b; i < e; ++i) f(i, tid);
        }
    };
    if (p <= 1) {
        body(0);
        return;
    }
    run_ranks(p, body);
}

// An allocator whose value-initialisation leaves trivial elements
// uninitialised: resize() of a raw_vector only reserves the pages, which the
// caller then fills (a parallel first touch, a copy from the device).
template <class T>
struct NoInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = NoInitAlloc<U>;
    };
    NoInitAlloc() = default;
    template <class U>
    NoInitAlloc(const NoInitAlloc<U> &) noexcept {}
    template <class U>
    void construct(U *p) noexcept {
        ::new (static_cast<void *>(p)) U;
    }
    template <class U, class... A>
    void construct(U *p, A &&...a) {
        ::new (static_cast<void *>(p)) U(std::forward<A>(a)...);
    }
};
template <class T>
using raw_vector = std::vector<T, NoInitAlloc<T>>;

// Copy n trivially copyable elements with up to nthreads threads, one piece
// of at least 4M elements each (each thread also takes the first touch of
// its piece of dst).
template <class T>
void parallel_copy(T *dst, const T *src, int64_t n, int nthreads) {
    const int p = int(std::min<int64_t>(nthreads, std::max<int64_t>(1, n >> 22)));
    parallel_for(p, p, [&](int64_t b, int64_t e, int) {
        for (int64_t i = b; i < e; ++i) {
            const int64_t lo = n * i / p, hi = n * (i + 1) / p;
            if (hi > lo) std::memcpy(static_cast<void *>(dst + lo), src + lo, size_t(hi - lo) * sizeof(T));
        }
    });
}

}  // namespace gale
