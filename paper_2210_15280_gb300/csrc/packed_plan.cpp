// packed_plan.cpp -- host-side row schedules of the packed substitution
// kernels (packed.h).
//
// Rows and their natural order.  Row (y, z) of the interior, y, z >= 1,
// y + z <= N - 2, has n = N - 1 - y - z points.  In the forward substitution
// (Alg. 2) its point x lies on hyperplane x + 2y + 3z, so the row's first
// point is on 1 + 2y + 3z and every later point one hyperplane further; the
// lower neighbours of a point lie in rows (y-1, z) (s, se), (y, z-1) (bc, be)
// and (y+1, z-1) (bnw, bn), whose first hyperplanes are 2, 3 and 1 earlier.
//
// Forward schedule.  Rows sorted by natural first hyperplane go, one by one,
// to the lane that is free first; the row starts at its natural hyperplane
// plus the current delay, or later if its lane is still busy, and the delay
// grows to match.  Delays never decrease along the order, so a producer row
// (always earlier in the order) has at most the delay of its consumer: every
// value is produced at an earlier step than the step that reads it.
//
// Backward schedule.  The same assignment run backwards: forward step tau is
// backward step T - 1 - tau (T rounded up to whole four-step blocks).  A row
// of n points on forward steps [s, s+n-1] covers backward steps
// [T - s - n, T - 1 - s], its point x at backward step T - s - x.  The upper neighbours of a point are the points that read it in
// the forward pass, so they were computed later there and come earlier here.
//
// Spacing on a lane.  Before each row the lane has one idle step (it switches
// to the row there), and the copy of the following row's coefficients and
// schedule entry, issued at the end of a row's first step, needs
// kPackedPre + 1 steps: consecutive rows A, B of a lane keep
//     s_B >= s_A + n_A + 1,  s_B >= s_A + kPackedPre + 2          (forward)
//     s_B + n_B >= s_A + n_A + kPackedPre + 2                      (backward,
// where B comes first and its first backward step is T - s_B - n_B).
#include <algorithm>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <string>
#include <vector>

#include "grid.h"
#include "packed.h"

namespace ilu {

bool make_packed_plan(int N, int lanes, PackedPlan *out, std::string *err) {
  if (N < 4 || N > 256 || lanes < 1 || lanes > 511) {
    *err = "packed schedule: bad size";
    return false;
  }
  struct Row {
    int st, y, z, n;
  };
  std::vector<Row> rows;
  rows.reserve((size_t)num_rows(N));
  for (int z = 1; z <= N - 3; ++z)
    for (int y = 1; y <= N - 2 - z; ++y) rows.push_back({1 + 2 * y + 3 * z, y, z, N - 1 - y - z});
  std::stable_sort(rows.begin(), rows.end(), [](const Row &a, const Row &b) { return a.st < b.st; });
  const int64_t R = num_rows(N);
  std::vector<int> t_of(R, -1), lane_of(R, -1), yz_of(R, 0);  // first step, lane, y | z << 16 (by row_id)
  for (const Row &r : rows) yz_of[row_id(N, r.y, r.z)] = r.y | (r.z << 16);
  using Free = std::pair<int, int>;  // (first step the lane could take, lane)
  std::priority_queue<Free, std::vector<Free>, std::greater<Free>> freeq;
  for (int l = 0; l < lanes; ++l) freeq.push({1, l});
  std::vector<int> last_t(lanes, -1), last_n(lanes, 0);  // the lane's previous row
  std::vector<std::vector<int>> per_lane(lanes);
  int delay = 0, T = 0;
  for (const Row &r : rows) {
    const Free f = freeq.top();
    freeq.pop();
    const int l = f.second;
    int t = std::max(r.st + delay, f.first);
    if (last_t[l] >= 0) t = std::max(t, last_t[l] + last_n[l] + kPackedPre + 2 - r.n);  // backward spacing
    delay = t - r.st;
    const int64_t id = row_id(N, r.y, r.z);
    t_of[id] = t;
    lane_of[id] = l;
    per_lane[l].push_back((int)id);
    last_t[l] = t;
    last_n[l] = r.n;
    freeq.push({t + std::max(r.n + 1, kPackedPre + 2), l});
    T = std::max(T, t + r.n + 1);  // one idle step after the last point: every backward first step >= 1
  }
  // producer code of (qy, qz) for consumer (y, z): the first value the
  // consumer reads at a step is written k0 = (first step of the consumer) -
  // (first step of the producer) + c steps earlier
  auto code = [&](int y, int z, int qy, int qz, int c, bool fwd, int *out_code) -> bool {
    if (qy < 1 || qz < 1 || qy + qz > N - 2) {
      *out_code = prod_code(kProdNone, 0, 0);
      return true;
    }
    const int64_t q = row_id(N, qy, qz), r = row_id(N, y, z);
    const int nq = N - 1 - qy - qz, nr = N - 1 - y - z;
    const int sr = fwd ? t_of[r] : T - t_of[r] - nr, sq = fwd ? t_of[q] : T - t_of[q] - nq;
    const int k0 = sr - sq + c;
    if (k0 < 2) return false;  // the first value would not be ready
    if (k0 >= (1 << 21)) return false;
    *out_code = prod_code(k0 <= kPackedRing - 1 ? kProdRing : kProdGlobal, lane_of[q], k0);
    return true;
  };
  T = (T + 3) & ~3;  // whole four-step blocks of the packed array
  out->N = N;
  out->lanes = lanes;
  out->nsteps = T;
  out->fwd.clear();
  out->bwd.clear();
  out->fwd.reserve((size_t)R);
  out->bwd.reserve((size_t)R);
  out->lane_off.assign((size_t)lanes + 1, 0);
  out->row_map.assign((size_t)R, 0);
  for (int l = 0; l < lanes; ++l) {
    out->lane_off[l] = (int)out->fwd.size();
    const std::vector<int> &ids = per_lane[l];
    for (size_t k = 0; k < ids.size(); ++k) {
      for (int pass = 0; pass < 2; ++pass) {
        const bool fwd = pass == 0;
        const int id = fwd ? ids[k] : ids[ids.size() - 1 - k];  // backward: the lane's rows in reverse
        const int y = yz_of[id] & 0xffff, z = yz_of[id] >> 16, n = N - 1 - y - z;
        int c[3];
        const bool ok = fwd ? code(y, z, y - 1, z, 0, true, &c[0]) && code(y, z, y, z - 1, 0, true, &c[1]) &&
                                  code(y, z, y + 1, z - 1, 1, true, &c[2])
                            : code(y, z, y + 1, z, 1, false, &c[0]) && code(y, z, y, z + 1, 1, false, &c[1]) &&
                                  code(y, z, y - 1, z + 1, 1, false, &c[2]);
        if (!ok) {
          *err = "packed schedule: a producer value is not ready in time";
          return false;
        }
        const int start = fwd ? t_of[id] : T - t_of[id] - n;
        int far = 0;  // some producer read back from global memory
        for (int j = 0; j < 3; ++j) far |= ((c[j] >> 30) & 3) == kProdGlobal;
        (fwd ? out->fwd : out->bwd)
            .push_back({start, n | (y << 10) | (z << 20), (int)grid_index(N, 0, y, z), id, {c[0], c[1], c[2]}, far});
      }
      out->row_map[ids[k]] = t_of[ids[k]] | (l << 20);
    }
  }
  out->lane_off[lanes] = (int)out->fwd.size();
  if ((int64_t)out->fwd.size() != R || T >= (1 << 20)) {
    *err = "packed schedule: rows lost or too many steps";
    return false;
  }
  return true;
}

const PackedPlan *packed_plan_cached(int N, std::string *err) {
  static std::mutex mu;
  static std::map<int, std::unique_ptr<PackedPlan>> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto &slot = cache[N];
  if (!slot) {
    auto p = std::make_unique<PackedPlan>();
    if (!make_packed_plan(N, kPackedLanes, p.get(), err)) return nullptr;
    slot = std::move(p);
  }
  return slot.get();
}

}  // namespace ilu
