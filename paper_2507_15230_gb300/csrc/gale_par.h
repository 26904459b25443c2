// Host thread-parallel loops shared by the host-side parts of the library
// (internal).
#pragma once

#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

namespace gale {

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
    std::vector<std::thread> th;
    th.reserve(p);
    for (int i = 0; i < p; ++i) {
        const int64_t b = n * i / p, e = n * (i + 1) / p;
        th.emplace_back([&f, b, e, i] { f(b, e, i); });
    }
    for (auto &t : th) t.join();
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
    std::vector<std::thread> th;
    for (int i = 0; i < p; ++i) th.emplace_back(body, i);
    for (auto &t : th) t.join();
}

}  // namespace gale
