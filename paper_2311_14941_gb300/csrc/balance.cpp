// balance.cpp -- load balancing of chemistry cells between processes (Sec. 2.5).
//
// The paper's solver redistributes the chemistry work between MPI ranks before every chemistry step so
// that all ranks carry about the same load.  Here the decision is one deterministic host computation
// over all ranks' per-cell costs (each rank runs it on the same all-gathered input and obtains the same
// plan; the cell states then move with one all-to-all and come back with another).
//
// Rule.  target = total cost / ranks.  Each rank keeps its cheapest cells (ascending cost, ties by local
// index) as long as their running sum stays within the target: the most cells a rank can keep without
// exceeding it, so the fewest cells move.  The other cells form a pool that is dealt in descending cost
// (ties by rank, then local index) to whichever rank currently has the least load (ties to the lowest
// rank).  Every such assignment goes to a rank at or below the target (the least current load never
// exceeds the mean of the current loads, which is at most the target), so no rank ends above
// target + the largest single cost, and a rank at or below the target moves none of its cells.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <queue>
#include <string>
#include <vector>

#include "compile.h"

namespace chemgb {

chem_status balance_plan(int world, const int64_t* counts, const double* costs, int32_t* dest, std::string& err) {
  if (world < 1) { err = "world must be >= 1"; return CHEM_EINVAL; }
  if (!counts) { err = "counts must not be NULL"; return CHEM_EINVAL; }
  std::vector<int64_t> first(world + 1, 0);
  for (int r = 0; r < world; ++r) {
    if (counts[r] < 0) { err = "counts[" + std::to_string(r) + "] is negative"; return CHEM_EINVAL; }
    first[r + 1] = first[r] + counts[r];
  }
  const int64_t N = first[world];
  if (N == 0) return CHEM_OK;
  if (!costs || !dest) { err = "costs and dest must not be NULL when there are cells"; return CHEM_EINVAL; }
  double total = 0.0;
  for (int64_t c = 0; c < N; ++c) {
    if (!std::isfinite(costs[c]) || costs[c] < 0.0) {
      err = "cost of cell " + std::to_string(c) + " is negative or not finite";
      return CHEM_EINVAL;
    }
    total += costs[c];
  }
  const double target = total / world;
  std::vector<double> load(world, 0.0);
  std::vector<int64_t> pool;                 // global cell numbers (rank-major)
  std::vector<int64_t> idx;
  for (int r = 0; r < world; ++r) {
    const int64_t b = first[r], n = counts[r];
    idx.resize(n);
    std::iota(idx.begin(), idx.end(), b);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return costs[x] < costs[y]; });
    double sum = 0.0;
    int64_t k = 0;
    for (; k < n; ++k) {
      const double s = sum + costs[idx[k]];
      if (s > target) break;
      sum = s;
      dest[idx[k]] = r;
    }
    load[r] = sum;
    pool.insert(pool.end(), idx.begin() + k, idx.end());
  }
  // descending cost; equal costs keep rank-major, index-ascending order
  std::stable_sort(pool.begin(), pool.end(), [&](int64_t x, int64_t y) { return costs[x] > costs[y]; });
  using Entry = std::pair<double, int>;      // (load, rank): smallest load first, then lowest rank
  std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> heap;
  for (int r = 0; r < world; ++r) heap.push({load[r], r});
  for (int64_t c : pool) {
    const Entry e = heap.top();
    heap.pop();
    dest[c] = e.second;
    heap.push({e.first + costs[c], e.second});
  }
  return CHEM_OK;
}

}  // namespace chemgb
