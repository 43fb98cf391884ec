// Host worker threads for the O(nnz) passes of problem creation and of the
// device layout build.
#pragma once

#include <algorithm>
#include <cstddef>
#include <exception>
#include <thread>
#include <vector>

namespace gb300lp {

// Run f(t, lo, hi) for t = 0 .. nt-1 over contiguous chunks [lo, hi) of
// [0, count), on up to 16 threads when `parallel` (else one call on the
// calling thread); nt is the number of chunks.  f must touch disjoint data
// per chunk and must not throw.  A thread that cannot be started runs its
// chunk on the calling thread; all are joined before this returns.
template <class F>
void host_parallel_chunks(size_t count, bool parallel, F f) {
  const unsigned nt =
      parallel && count > 0 ? std::min(16u, std::max(1u, std::thread::hardware_concurrency())) : 1u;
  if (nt <= 1) {
    f(0u, (size_t)0, count);
    return;
  }
  std::vector<std::thread> ts;
  ts.reserve(nt);
  for (unsigned t = 0; t < nt; ++t) {
    const size_t lo = count * t / nt, hi = count * (t + 1) / nt;
    try {
      ts.emplace_back(f, t, lo, hi);
    } catch (const std::exception &) {
      f(t, lo, hi);
    }
  }
  for (std::thread &th : ts)
    if (th.joinable()) th.join();
}

}  // namespace gb300lp
