// shard.cpp -- the split of a set of macro-tetrahedra over several GPUs
// (ilu_partition).  Host code only.
//
// Interior solves on different macro-tetrahedra are independent (the hybrid
// grid of Sec. 2.1 couples them only through the interface data, which the
// interior smoother reads and never writes), so a batch or a stream of
// requests shards by tet with no exchange between GPUs.  The split is the
// longest-processing-time rule: tets in decreasing order of cost, each to the
// GPU with the least cost so far (ties to the lower rank, equal costs in
// index order), which keeps the largest load within 4/3 of the optimum.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/ilu.h"

namespace ilu {
void set_last_error(const std::string &msg);
}

extern "C" ilu_status ilu_partition(int n, const double *cost, int nranks, int *rank_of, double *load) {
  if (n < 0 || nranks < 1 || (n > 0 && (!cost || !rank_of))) {
    ilu::set_last_error("ilu_partition: bad argument");
    return ILU_EINVAL;
  }
  for (int i = 0; i < n; ++i)
    if (!(cost[i] >= 0.0) || !std::isfinite(cost[i])) {
      ilu::set_last_error("ilu_partition: costs must be finite and non-negative");
      return ILU_EINVAL;
    }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> sum(nranks, 0.0);
  for (int i : order) {
    const int r = (int)(std::min_element(sum.begin(), sum.end()) - sum.begin());
    rank_of[i] = r;
    sum[r] += cost[i];
  }
  if (load) std::copy(sum.begin(), sum.end(), load);
  return ILU_OK;
}
