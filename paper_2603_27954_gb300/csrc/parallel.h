// Host-side parallel loop for the mesh build: the index range is cut into
// contiguous chunks handed to std::threads.  Every caller writes results
// indexed by the loop variable only, so the output does not depend on the
// thread count or the schedule.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <exception>
#include <mutex>
#include <thread>
#include <vector>

namespace lbm {

inline int host_threads() {
  static const int n = [] {
    if (const char* e = std::getenv("LBM_HOST_THREADS")) {
      int v = std::atoi(e);
      if (v > 0) return std::min(v, 256);
    }
    unsigned h = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(h, 64u));
  }();
  return n;
}

// f(i) for i in [0, n); chunks of `grain` indices are claimed dynamically.
// An exception thrown by f on any thread stops the loop and is rethrown on
// the calling thread once every thread has finished (none escapes a worker,
// which would end the process); if a thread cannot be started, the threads
// already running finish the loop.
template <class F>
void parallel_for(long long n, F&& f, long long grain = 1) {
  const int nt = (int)std::min<long long>(host_threads(), (n + grain - 1) / std::max(1LL, grain));
  if (nt <= 1) {
    for (long long i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<long long> next{0};
  std::exception_ptr err;
  std::mutex err_mu;
  auto work = [&] {
    try {
      for (;;) {
        const long long b = next.fetch_add(grain);
        if (b >= n) break;
        const long long e = std::min(n, b + grain);
        for (long long i = b; i < e; ++i) f(i);
      }
    } catch (...) {
      std::lock_guard<std::mutex> lock(err_mu);
      if (!err) err = std::current_exception();
      next.store(n);
    }
  };
  std::vector<std::thread> pool;
  pool.reserve(nt - 1);
  try {
    for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  } catch (...) {
    // fewer threads: the ones started and this one finish the loop
  }
  work();
  for (auto& th : pool) th.join();
  if (err) std::rethrow_exception(err);
}

// ascending sort: chunks sorted in parallel, then merged pairwise
template <class T>
void parallel_sort(std::vector<T>& v) {
  const long long n = (long long)v.size();
  const int chunks = (int)std::min<long long>(host_threads(), std::max(1LL, n / 65536));
  if (chunks <= 1) {
    std::sort(v.begin(), v.end());
    return;
  }
  std::vector<long long> cut(chunks + 1);
  for (int c = 0; c <= chunks; ++c) cut[c] = n * c / chunks;
  parallel_for(chunks, [&](long long c) { std::sort(v.begin() + cut[c], v.begin() + cut[c + 1]); });
  for (int w = 1; w < chunks; w *= 2) {
    std::vector<long long> merges;
    for (int c = 0; c + w < chunks; c += 2 * w) merges.push_back(c);
    parallel_for((long long)merges.size(), [&](long long k) {
      const int c = (int)merges[k];
      const int e = std::min(chunks, c + 2 * w);
      std::inplace_merge(v.begin() + cut[c], v.begin() + cut[c + w], v.begin() + cut[e]);
    });
  }
}

}  // namespace lbm
