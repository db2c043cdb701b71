// Host-side data parallelism for the hierarchy construction and symbolic
// analysis: [0, n) split into contiguous chunks, one worker thread each.
// Callers write only the outputs of their own chunk and merge chunk results
// in chunk order, so every result is independent of the thread count.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <exception>
#include <thread>
#include <vector>

namespace hsim {

// Worker threads for host loops: HSIM_HOST_THREADS if set (>= 1), else the
// hardware concurrency, at most 64.
inline int host_threads() {
    static const int t = [] {
        const char *e = std::getenv("HSIM_HOST_THREADS");
        long v = e ? std::strtol(e, nullptr, 10) : 0;
        if (v < 1) v = (long)std::thread::hardware_concurrency();
        return (int)std::min<long>(std::max<long>(v, 1), 64);
    }();
    return t;
}

// Number of chunks parallel_chunks uses for n items of at least min_chunk each.
inline int chunk_count(int64_t n, int64_t min_chunk) {
    const int64_t by_size = std::max<int64_t>(1, n / std::max<int64_t>(1, min_chunk));
    return (int)std::min<int64_t>(host_threads(), by_size);
}

// f(chunk, begin, end) for the chunks [begin, end) of [0, n), chunk =
// 0..chunk_count(n, min_chunk)-1, concurrently.  An exception thrown by any
// chunk is rethrown here (the first in chunk order) after all have finished.
template <class F>
void parallel_chunks(int64_t n, int64_t min_chunk, F &&f) {
    const int t = chunk_count(n, min_chunk);
    if (t <= 1) {
        f(0, (int64_t)0, n);
        return;
    }
    std::vector<std::exception_ptr> err(t);
    std::vector<std::thread> th;
    th.reserve(t);
    for (int c = 0; c < t; ++c) {
        const int64_t b = n * c / t, e = n * (c + 1) / t;
        th.emplace_back([&f, &err, c, b, e] {
            try {
                f(c, b, e);
            } catch (...) {
                err[c] = std::current_exception();
            }
        });
    }
    for (auto &x : th) x.join();
    for (auto &e : err)
        if (e) std::rethrow_exception(e);
}

}  // namespace hsim
