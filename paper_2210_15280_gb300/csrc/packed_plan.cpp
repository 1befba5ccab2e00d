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
// Forward schedule (list scheduling).  A row is ready once its producers
// have starts; it may start q + 1 - c steps after each producer starts (c = 1
// for (y+1, z-1), whose first hyperplane is one earlier, else 0), which puts
// every value it reads at least q steps before the step that reads it: the
// kernels meet at a block barrier only every q steps, after steps q - 1
// (mod q), so a value is visible to every lane q steps after it was written
// at the latest.  Ready rows, earliest allowed start first (ties: natural
// first hyperplane), go to the lane that frees up first, and start when both
// are ready.  Starts are multiples of the quantum q and rows take
// ceil(n / q) * q steps (the last ones idle), so that a lane changes rows only
// on steps q - 1 (mod q) in both passes: the kernels test for that only
// there.  q is 1 up to level 6 (where the dependency depth sets the step
// count, and a larger q would lengthen it), 2 at level 7 and 4 at level 8
// (where the lanes' total work does).
//
// Backward schedule.  The same assignment run backwards: forward step tau is
// backward step T - 1 - tau (T rounded up to whole kPackedBlock-step
// blocks).  A row of n points (n' padded) on forward steps [s, s+n'-1]
// covers backward steps [T - s - n', T - 1 - s], its point x at backward
// step T - s - x.  The upper neighbours of a point are the points that read
// it in the forward pass, so they were computed later there and come earlier
// here.
//
// Spacing on a lane.  Before each row the lane has one step without a point
// (it switches to the row there), and so has every step after a row's last
// point.  The copy of a row's coefficients and of the schedule entry after
// it is issued kPackedPre steps before the row's switch step, when the stage
// is free: the previous row's switch read it at least a step earlier.  So
// consecutive rows A, B of a lane (padded lengths n'_A, n'_B) keep
//     s_B >= s_A + n'_A + 1,  s_B >= s_A + kPackedPre + 2          (forward)
//     s_B + n'_B >= s_A + n'_A + kPackedPre + 2                    (backward,
// where B comes first and switches at T - s_B - n'_B - 1).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <string>
#include <tuple>
#include <vector>

#include "grid.h"
#include "packed.h"

namespace ilu {

int packed_quantum(int N) { return N <= 64 ? 1 : (N <= 128 ? 2 : 4); }
int packed_cluster(int N) { return N <= 128 ? 1 : 2; }
int packed_lanes(int N) { return packed_cluster(N) == 1 ? kPackedLanes : 2 * kPackedClusterLanes; }

bool make_packed_plan(int N, int lanes, int q, PackedPlan *out, std::string *err) {
  // lanes <= 1016: every ring word (below 32 rows of lanes + 8 words) fits 15 bits
  if (N < 4 || N > 256 || lanes < 1 || lanes > 1016 || (q != 1 && q != 2 && q != 4)) {
    *err = "packed schedule: bad size";
    return false;
  }
  const int64_t R = num_rows(N);
  std::vector<int> y_of(R), z_of(R), n_of(R), nat(R), pending(R, 0);
  std::vector<std::vector<int>> cons(R);
  auto rid = [&](int y, int z) -> int64_t {
    return (y >= 1 && z >= 1 && y + z <= N - 2) ? row_id(N, y, z) : -1;
  };
  // forward producers of row (y, z) and their c (the first value a consumer
  // reads at a step is the producer's value c steps after the one at the
  // consumer's own x)
  const int pdy[3] = {-1, 0, 1}, pdz[3] = {0, -1, -1}, pc[3] = {0, 0, 1};
  for (int z = 1; z <= N - 3; ++z)
    for (int y = 1; y <= N - 2 - z; ++y) {
      const int64_t id = row_id(N, y, z);
      y_of[id] = y;
      z_of[id] = z;
      n_of[id] = N - 1 - y - z;
      nat[id] = 1 + 2 * y + 3 * z;
      for (int j = 0; j < 3; ++j) {
        const int64_t p = rid(y + pdy[j], z + pdz[j]);
        if (p >= 0) {
          ++pending[id];
          cons[p].push_back((int)id);
        }
      }
    }
  // list schedule: ready rows by earliest start, then natural hyperplane
  using Ready = std::tuple<int, int, int>;  // (earliest start, natural first hyperplane, row)
  std::priority_queue<Ready, std::vector<Ready>, std::greater<Ready>> ready;
  for (int64_t id = 0; id < R; ++id)
    if (pending[id] == 0) ready.push({1, nat[id], (int)id});
  using Free = std::pair<int, int>;  // (first step the lane could take a row at, lane)
  std::priority_queue<Free, std::vector<Free>, std::greater<Free>> freeq;
  for (int l = 0; l < lanes; ++l) freeq.push({1, l});
  std::vector<int> s_of(R, -1), lane_of(R, -1), last_s(lanes, -1), last_np(lanes, 0);
  std::vector<std::vector<int>> per_lane(lanes);
  auto padded = [&](int n) { return (n + q - 1) / q * q; };
  int T = 0, done = 0;
  while (!ready.empty()) {
    const Ready rd = ready.top();
    ready.pop();
    const int id = std::get<2>(rd);
    const Free f = freeq.top();
    freeq.pop();
    const int l = f.second, np = padded(n_of[id]);
    int s = std::max(std::get<0>(rd), f.first);
    if (last_s[l] >= 0)
      s = std::max({s, last_s[l] + last_np[l] + 1, last_s[l] + kPackedPre + 2,
                    last_s[l] + last_np[l] + kPackedPre + 2 - np});
    s = (s + q - 1) / q * q;
    s_of[id] = s;
    lane_of[id] = l;
    per_lane[l].push_back(id);
    last_s[l] = s;
    last_np[l] = np;
    freeq.push({s + np + 1, l});
    T = std::max(T, s + np + 1);  // an idle step after the last row: every backward switch step >= 0
    ++done;
    for (int c : cons[id])
      if (--pending[c] == 0) {
        int e = 1;
        for (int j = 0; j < 3; ++j) {
          const int64_t p = rid(y_of[c] + pdy[j], z_of[c] + pdz[j]);
          if (p >= 0) e = std::max(e, s_of[p] + q + 1 - pc[j]);
        }
        ready.push({e, nat[c], c});
      }
  }
  T = (T + kPackedBlock - 1) / kPackedBlock * kPackedBlock;  // whole blocks of the kernels' loop
  if (done != R || T >= (1 << 16) || R >= (1 << 15)) {  // the limits of the entries' fields
    *err = "packed schedule: rows lost or too many steps";
    return false;
  }
  // first point of row r in a pass (backward: the forward schedule reversed in time)
  auto first = [&](int64_t r, bool fwd) { return fwd ? s_of[r] : T - s_of[r] - n_of[r]; };
  out->N = N;
  out->lanes = lanes;
  out->q = q;
  out->nsteps = T;
  out->fwd.clear();
  out->bwd.clear();
  out->fwd.reserve((size_t)R);
  out->bwd.reserve((size_t)R);
  out->lane_off.assign((size_t)lanes + 1, 0);
  out->row_map.assign((size_t)R, 0);
  const double hh = 0.5 / N;
  // the kernels meet at a block barrier every q steps, so lanes can be up to
  // q - 1 steps apart: a value read from the ring must not be overwritten by
  // then (k0 <= kPackedRing + 1 - q)
  const int ring_max = std::min(kPackedRing - 1, kPackedRing + 1 - q);
  const int RW = packed_ring_row(lanes);
  for (int l = 0; l < lanes; ++l) {
    out->lane_off[l] = (int)out->fwd.size();
    const std::vector<int> &ids = per_lane[l];
    for (size_t k = 0; k < ids.size(); ++k) {
      for (int pass = 0; pass < 2; ++pass) {
        const bool fwd = pass == 0;
        const int id = fwd ? ids[k] : ids[ids.size() - 1 - k];  // backward: the lane's rows in reverse
        const int y = y_of[id], z = z_of[id], n = n_of[id], np = padded(n);
        const int lo = first(id, fwd);
        const int sw = fwd ? s_of[id] - 1 : T - s_of[id] - np - 1;  // a multiple of q, minus 1
        const int tau0 = sw & ~(kPackedBlock - 1);
        int code[3], R3[3], gm = 0;
        for (int j = 0; j < 3; ++j) {
          // producers: forward (y-1, z), (y, z-1), (y+1, z-1); backward (y+1, z), (y, z+1), (y-1, z+1)
          const int64_t p = fwd ? rid(y + pdy[j], z + pdz[j]) : rid(y - pdy[j], z - pdz[j]);
          if (p < 0) {
            code[j] = prod_code(kProdNone, 0, 0);
            R3[j] = lanes;  // the ring column nothing writes
            continue;
          }
          const int k0 = lo - first(p, fwd) + (fwd ? pc[j] : 1);
          if (k0 < q + 1 || k0 >= (1 << 21)) {
            *err = "packed schedule: a producer value is not ready in time";
            return false;
          }
          const bool ring = k0 <= ring_max;
          // a queue producer's values are read back at steps sw + 1 - k0 ..
          // lo + n - k0 of the pass: they must lie in the packed array
          if (!ring && (sw + 1 - k0 < 0 || lo + n - k0 > T - 1)) {
            *err = "packed schedule: a far producer value outside the packed array";
            return false;
          }
          code[j] = prod_code(ring ? kProdRing : kProdGlobal, lane_of[p], k0);
          R3[j] = ring ? ((tau0 + 1 - k0) & (kPackedRing - 1)) * RW + lane_of[p] : lanes;
          gm |= ring ? 0 : 1 << j;
        }
        const int K = N - y - z, xsw = fwd ? 0 : n + lo - sw;
        const float tt0 = (float)((double)(2 * xsw - K) * hh);
        PackedEntry e;
        e.sw_dlo_far = sw | ((lo - sw) << 16) | (gm << 20);
        e.nyz = n | (y << 10) | (z << 20);
        e.r01 = R3[0] | (R3[1] << 15);
        e.r2rid = R3[2] | (id << 15);
        std::memcpy(&e.tt0, &tt0, sizeof(float));
        for (int j = 0; j < 3; ++j) e.p[j] = code[j];
        (fwd ? out->fwd : out->bwd).push_back(e);
      }
      out->row_map[ids[k]] = s_of[ids[k]] | (l << 20);
    }
  }
  out->lane_off[lanes] = (int)out->fwd.size();
  if ((int64_t)out->fwd.size() != R) {
    *err = "packed schedule: rows lost";
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
    if (!make_packed_plan(N, packed_lanes(N), packed_quantum(N), p.get(), err)) return nullptr;
    slot = std::move(p);
  }
  return slot.get();
}

}  // namespace ilu
