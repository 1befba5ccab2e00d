// batch.cu -- many macro-tetrahedra smoothed together (ilu_batch_*).
//
// A pass over the batch (one sweep of Alg. 2 on every tet) is
//   1. one reset of all progress words and ticket counters,
//   2. one residual launch covering every tet (1-D grid, per-tet block ranges),
//   3. the substitutions, as independent branches of the pass so that their
//      kernels run concurrently:
//      - tets whose handles use the packed kernels: one launch per row-table
//        layout and schedule quantum (level 7 and level 8 schedules differ),
//        a CTA (level 8: a cluster of two) per tet holding its forward and
//        backward substitution, tets ordered by their step count, longest
//        first; no CTA waits on another.  The launches follow one another
//        on the pass's stream, the group with the longest tets first, each
//        later one a programmatic dependent of the one before: its CTAs are
//        dispatched once every CTA of the longer group has started, so the
//        short tets fill the SMs the long ones leave free and never hold an
//        SM that a long tet's cluster waits for;
//      - the other tets, grouped by level and row-polynomial layout: one
//        forward and one backward slab launch per group.  Inside a group the
//        clusters of every tet take tickets tet by tet, in dependency order
//        within a tet, so any cluster waits only on clusters that took earlier
//        tickets and are therefore resident or finished: the launch cannot
//        deadlock whatever the residency.
// A tet whose row degree is below its launch's register degree evaluates
// zero leading coefficients, which leaves its results bit for bit those of
// its own launch.  The autotuner times the slab partitions (packed tets have
// no partition to choose).
//
// The passes of one ilu_batch_smooth call are captured once into a CUDA graph
// (re-captured when `sweeps` changes) and replayed on the caller's stream.
// The batch reuses each tet's scratch vector and tables: a tet must not be
// smoothed through its own handle or another batch while a batch call on it
// runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ilu.h"
#include "hooks.h"
#include "kernels.cuh"

using namespace ilu;

namespace ilu {
void set_last_error(const std::string &msg);
}

namespace {

ilu_status fail(ilu_status s, const std::string &msg) {
  set_last_error(msg);
  return s;
}

#define BK(call, what)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(ILU_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr long long kBatchSpins = 4000000;

struct Group {
  int N = 0, reg = -1, dxp = 0;
  std::vector<int> members;  // tet indices, in ticket order
  WaveLaunch wl = {};
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
};

// Tets on the packed kernels with the same row-table layout and schedule
// quantum: one launch, a CTA (or cluster) per tet, longest tets first (their
// CTAs start first).
struct PackedGroup {
  int N = 0, dxp = 0, reg = 0, q = 1, cl = 1;
  bool v1 = false;
  std::vector<int> members;  // tet indices, most steps first
  PackedLaunch pl = {};
  cudaEvent_t done = nullptr;  // after the launch: joins it to the update
};

}  // namespace

struct ilu_batch_s {
  int device = 0, precision = 0, kind = 0, n = 0;
  long long max_spins = kBatchSpins;
  bool failed = false;
  std::vector<ilu_tet> tets;
  std::vector<TetView> views;
  std::vector<DevTet> dev;  // host copies of d_tets
  std::vector<Group> groups;
  std::vector<PackedGroup> pgroups;
  int *d_porder = nullptr;  // tet order of the packed launches
  int2 *d_rmap = nullptr;  // per operator kind: (tet, its block) of each block of its residual launch
  int rblocks[3] = {0, 0, 0};
  size_t rat[3] = {0, 0, 0};
  int total_blocks = 0, nflags = 0;
  DevTet *d_tets = nullptr;
  int2 *d_iomap = nullptr;  // (tet, its block) of each block of the update launch
  int *d_maps = nullptr, *d_flags = nullptr;
  void **d_ptrs = nullptr;  // xs[n] then bs[n]
  void **h_ptrs = nullptr;  // pinned staging of the pointer arrays
  cudaEvent_t ptr_ev = nullptr, fork = nullptr;
  LaunchStatus *d_status = nullptr, *h_status = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_sweeps = 0;
  int tuned_zb = 0;  // autotuner's choice (0: not tuned)
  int explicit_slabs = 0;
  bool tuned_largest = false;
  double tuned_ms = -1;
};

namespace {

// device state of one launch plan (rebuilt while autotuning)
void free_plan(ilu_batch b) {
  cudaSetDevice(b->device);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->graph_sweeps = 0;
  for (auto &g : b->groups) {
    if (g.st) cudaStreamDestroy(g.st);
    if (g.done) cudaEventDestroy(g.done);
  }
  b->groups.clear();
  for (auto &g : b->pgroups)
    if (g.done) cudaEventDestroy(g.done);
  b->pgroups.clear();
  cudaFree(b->d_porder);
  b->d_porder = nullptr;
  cudaFree(b->d_rmap);
  b->d_rmap = nullptr;
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->ptr_ev) cudaEventDestroy(b->ptr_ev);
  if (b->fork) cudaEventDestroy(b->fork);
  b->cap = nullptr;
  b->ptr_ev = b->fork = nullptr;
  cudaFree(b->d_tets);
  cudaFree(b->d_iomap);
  cudaFree(b->d_maps);
  cudaFree(b->d_flags);
  cudaFree(b->d_ptrs);
  cudaFree(b->d_status);
  b->d_tets = nullptr;
  b->d_iomap = nullptr;
  b->d_maps = b->d_flags = nullptr;
  b->d_ptrs = nullptr;
  b->d_status = nullptr;
  if (b->h_ptrs) cudaFreeHost(b->h_ptrs);
  if (b->h_status) cudaFreeHost(b->h_status);
  b->h_ptrs = nullptr;
  b->h_status = nullptr;
}

void release(ilu_batch b) {
  if (!b) return;
  free_plan(b);
  delete b;
}

// Build groups, per-tet geometry and flag layout, device arrays and the
// launch shapes.  zb: layers per slab CTA (0: the single-tet default);
// largest: clusters as large as the device schedules (fewer slow hops
// between clusters), else the size with the most resident CTAs.
ilu_status build(ilu_batch b, int zb_pref, bool largest) {
  const int n = b->n;
  // groups keyed by (level, polynomial class, padded row length); classes:
  // rows in registers, rows in shared memory, tabulated values
  auto cls = [](const TetView &v) { return v.reg >= 0 ? 1 : (v.reg == kWaveTabulated ? 2 : 0); };
  std::map<std::tuple<int, int, int>, int> key;
  std::map<std::pair<int, int>, int> pkey;  // packed tets by table layout and start quantum (which
                                            // also fixes the cluster size)
  for (int i = 0; i < n; ++i) {
    const TetView &v = b->views[i];
    if (v.packed) {
      pkey.emplace(std::make_pair(v.rstride, v.packed_q), 0);
      continue;
    }
    const auto k = std::make_tuple(-v.N, cls(v), v.rstride);  // largest levels first
    auto it = key.find(k);
    if (it == key.end()) {
      it = key.emplace(k, 0).first;
    }
    (void)it;
  }
  int gi = 0;
  for (auto &kv : key) kv.second = gi++;
  b->groups.assign(key.size(), Group{});
  int pgi = 0;
  for (auto &kv : pkey) kv.second = pgi++;
  b->pgroups.assign(pkey.size(), PackedGroup{});
  for (int i = 0; i < n; ++i) {
    const TetView &v = b->views[i];
    if (v.packed) {
      PackedGroup &pg = b->pgroups[pkey[std::make_pair(v.rstride, v.packed_q)]];
      pg.N = std::max(pg.N, v.N);
      pg.dxp = v.rstride;
      pg.q = v.packed_q;
      pg.cl = v.packed_cl;
      pg.reg = v.dx <= 3 ? 3 : 6;  // the degree of the tets' packed tables (zero padded, as their own launches)
      pg.v1 = pg.v1 || v.dev->bnd != nullptr;
      pg.members.push_back(i);
      continue;
    }
    Group &g = b->groups[key[std::make_tuple(-v.N, cls(v), v.rstride)]];
    g.N = v.N;
    g.dxp = v.rstride;
    g.reg = v.reg >= 0 ? std::max(g.reg, v.reg) : v.reg;
    g.members.push_back(i);
  }
  // per-tet descriptors with geometry and progress words in the batch's flag array
  b->dev.resize(n);
  for (auto &pg : b->pgroups) {
    for (int i : pg.members) {
      DevTet d = *b->views[i].dev;
      d.fwd.P = d.bwd.P = 0;  // no slab launches, no progress words
      b->dev[i] = d;
    }
    std::stable_sort(pg.members.begin(), pg.members.end(),
                     [&](int a, int c) { return b->views[a].packed_steps > b->views[c].packed_steps; });
  }
  // the group with the largest level (the longest tets) launches first
  std::stable_sort(b->pgroups.begin(), b->pgroups.end(),
                   [](const PackedGroup &a, const PackedGroup &c) { return a.N > c.N; });
  int off = 0;
  for (auto &g : b->groups) {
    for (int i : g.members) {
      const TetView &v = b->views[i];
      DevTet d = *v.dev;
      const int layers = std::max(1, v.N - 3);
      const int requested = b->explicit_slabs > 0 ? b->explicit_slabs : (zb_pref > 0 ? (layers + zb_pref - 1) / zb_pref : 0);
      d.fwd = wave_geom(v.N, v.kind, v.rstride, v.reg, true, requested);
      d.bwd = wave_geom(v.N, v.kind, v.rstride, v.reg, false, requested);
      d.fwd.prog = off;
      d.bwd.prog = off + d.fwd.P;
      off += d.fwd.P + d.bwd.P;
      d.fwd.ticket = d.bwd.ticket = -1;  // batch launches count tickets in the group's counters
      b->dev[i] = d;
    }
  }
  const int ticket0 = off;
  b->nflags = off + 2 * (int)b->groups.size();
  // block maps of the residual and update launches: (tet, its block)
  std::vector<int2> iomap;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < residual_blocks(b->views[i].N); ++k) iomap.push_back(make_int2(i, k));
  b->total_blocks = (int)iomap.size();
  BK(cudaMalloc(&b->d_flags, sizeof(int) * b->nflags), "cudaMalloc flags");
  BK(cudaMemset(b->d_flags, 0, sizeof(int) * b->nflags), "cudaMemset flags");
  for (auto &d : b->dev) d.flags = b->d_flags;
  BK(cudaMalloc(&b->d_tets, sizeof(DevTet) * n), "cudaMalloc tets");
  BK(cudaMemcpy(b->d_tets, b->dev.data(), sizeof(DevTet) * n, cudaMemcpyHostToDevice), "upload tets");
  BK(cudaMalloc(&b->d_iomap, sizeof(int2) * std::max<size_t>(iomap.size(), 1)), "cudaMalloc block map");
  if (!iomap.empty())
    BK(cudaMemcpy(b->d_iomap, iomap.data(), sizeof(int2) * iomap.size(), cudaMemcpyHostToDevice), "upload block map");
  {  // residual launches by operator kind: the blocks of that kind's tets
    std::vector<int2> rmap;
    for (int op = 0; op < 3; ++op) {
      b->rat[op] = rmap.size();
      for (int i = 0; i < n; ++i)
        if (residual_op(b->dev[i]) == op) {
          const int nb = op == kOpConst ? residual_strip_blocks(b->views[i].N) : residual_blocks(b->views[i].N);
          for (int k = 0; k < nb; ++k) rmap.push_back(make_int2(i, k));
        }
      b->rblocks[op] = (int)(rmap.size() - b->rat[op]);
    }
    BK(cudaMalloc(&b->d_rmap, sizeof(int2) * std::max<size_t>(rmap.size(), 1)), "cudaMalloc residual maps");
    if (!rmap.empty())
      BK(cudaMemcpy(b->d_rmap, rmap.data(), sizeof(int2) * rmap.size(), cudaMemcpyHostToDevice),
         "upload residual maps");
  }
  BK(cudaMalloc(&b->d_ptrs, sizeof(void *) * 2 * n), "cudaMalloc pointer arrays");
  BK(cudaMemset(b->d_ptrs, 0, sizeof(void *) * 2 * n), "cudaMemset pointer arrays");
  BK(cudaMallocHost(&b->h_ptrs, sizeof(void *) * 2 * n), "cudaMallocHost pointer arrays");
  BK(cudaMalloc(&b->d_status, sizeof(LaunchStatus)), "cudaMalloc status");
  BK(cudaMemset(b->d_status, 0, sizeof(LaunchStatus)), "cudaMemset status");
  BK(cudaMallocHost(&b->h_status, sizeof(LaunchStatus)), "cudaMallocHost status");
  std::memset(b->h_status, 0, sizeof(LaunchStatus));
  // cluster maps: per group prefix_f (m+1), prefix_b (m+1), order (m)
  std::vector<int> maps;
  std::vector<size_t> map_at(b->groups.size());
  for (size_t g = 0; g < b->groups.size(); ++g) {
    Group &G = b->groups[g];
    WaveLaunch &L = G.wl;
    L = {};
    L.tets = b->d_tets;
    L.kind = b->kind;
    L.reg = G.reg;
    L.dxp = G.dxp;
    for (int i : G.members) {
      const DevTet &d = b->dev[i];
      const TetView &v = b->views[i];
      L.v1 = L.v1 || d.bnd != nullptr;
      L.block_f = std::max(L.block_f, (d.fwd.zb * d.fwd.wpl + 1) * 32);
      L.block_b = std::max(L.block_b, (d.bwd.zb * d.bwd.wpl + 1) * 32);
      L.smem_f = std::max(L.smem_f, wave_smem_bytes(v.N, d.fwd, b->kind, v.rstride, G.reg, true));
      L.smem_b = std::max(L.smem_b, wave_smem_bytes(v.N, d.bwd, b->kind, v.rstride, G.reg, false));
      L.maxP_f = std::max(L.maxP_f, d.fwd.P);
      L.maxP_b = std::max(L.maxP_b, d.bwd.P);
    }
    int qf[1 + kClusterCands] = {}, qb[1 + kClusterCands] = {};
    BK(launch_forward(L, nullptr, 0, nullptr, qf), "cluster query");
    BK(launch_backward(L, nullptr, 0, nullptr, qb), "cluster query");
    auto best = [largest](const int *q, int maxP) {
      if (largest) return q[0];
      int cs = 1, res = 0;
      for (int i = 0; i < kClusterCands; ++i) {
        const int c = std::min(kClusterSizes[i], maxP);
        if (q[1 + i] * c > res) {
          res = q[1 + i] * c;
          cs = c;
        }
      }
      return cs;
    };
    L.csize_f = best(qf, L.maxP_f);
    L.csize_b = best(qb, L.maxP_b);
    const size_t m = G.members.size();
    map_at[g] = maps.size();
    maps.push_back(0);
    for (int i : G.members) maps.push_back(maps.back() + (b->dev[i].fwd.P + L.csize_f - 1) / L.csize_f);
    L.clusters_f = maps.back();
    maps.push_back(0);
    for (int i : G.members) maps.push_back(maps.back() + (b->dev[i].bwd.P + L.csize_b - 1) / L.csize_b);
    L.clusters_b = maps.back();
    for (int i : G.members) maps.push_back(i);
    (void)m;
  }
  BK(cudaMalloc(&b->d_maps, sizeof(int) * std::max<size_t>(maps.size(), 1)), "cudaMalloc cluster maps");
  if (!maps.empty())
    BK(cudaMemcpy(b->d_maps, maps.data(), sizeof(int) * maps.size(), cudaMemcpyHostToDevice), "upload cluster maps");
  {
    std::vector<int> porder;
    for (auto &pg : b->pgroups) porder.insert(porder.end(), pg.members.begin(), pg.members.end());
    BK(cudaMalloc(&b->d_porder, sizeof(int) * std::max<size_t>(porder.size(), 1)), "cudaMalloc packed order");
    if (!porder.empty())
      BK(cudaMemcpy(b->d_porder, porder.data(), sizeof(int) * porder.size(), cudaMemcpyHostToDevice),
         "upload packed order");
    size_t at = 0;
    for (auto &pg : b->pgroups) {
      PackedLaunch &L = pg.pl;
      L.after_packed = &pg != &b->pgroups.front();
      L.tets = b->d_tets;
      L.order = b->d_porder + at;
      L.ntets = (int)pg.members.size();
      L.reg = pg.reg;
      L.q = pg.q;
      L.cl = pg.cl;
      L.v1 = pg.v1;
      at += pg.members.size();
      BK(cudaEventCreateWithFlags(&pg.done, cudaEventDisableTiming), "cudaEventCreate");
    }
  }
  for (size_t g = 0; g < b->groups.size(); ++g) {
    Group &G = b->groups[g];
    const int m = (int)G.members.size();
    const int *pf = b->d_maps + map_at[g], *pb = pf + m + 1, *order = pb + m + 1;
    G.wl.map_f = {pf, order, m, b->d_flags + ticket0 + 2 * (int)g, nullptr, nullptr};
    G.wl.map_b = {pb, order, m, b->d_flags + ticket0 + 2 * (int)g + 1, b->d_ptrs, nullptr};
    BK(cudaStreamCreateWithFlags(&G.st, cudaStreamNonBlocking), "cudaStreamCreate");
    BK(cudaEventCreateWithFlags(&G.done, cudaEventDisableTiming), "cudaEventCreate");
  }
  BK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "cudaStreamCreate");
  BK(cudaEventCreateWithFlags(&b->ptr_ev, cudaEventDisableTiming), "cudaEventCreate");
  BK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "cudaEventCreate");
  return ILU_OK;
}

// record `sweeps` passes on the capture stream (the groups fork and join)
ilu_status record_passes(ilu_batch b, int sweeps) {
  cudaStream_t s = b->cap;
  for (int k = 0; k < sweeps; ++k) {
    BK(cudaMemsetAsync(b->d_flags, 0, sizeof(int) * b->nflags, s), "reset flags");
    for (int op = 0; op < 3; ++op) {
      BK(launch_residual_batch(b->d_tets, b->d_rmap + b->rat[op], b->rblocks[op], b->kind, op,
                               b->d_ptrs, b->d_ptrs + b->n, s),
         "batched residual launch");
    }
    BK(cudaEventRecord(b->fork, s), "fork");
    // the packed groups on this stream, longest tets first, each later launch
    // a programmatic dependent of the one before; each launch's event joins
    // it to the update below, whatever the order in which they end
    for (auto &g : b->pgroups) {
      BK(launch_packed(g.pl, s), "packed substitution launch");
      BK(cudaEventRecord(g.done, s), "packed group end");
    }
    for (auto &g : b->groups) {
      BK(cudaStreamWaitEvent(g.st, b->fork, 0), "fork wait");
      BK(launch_forward(g.wl, b->d_status, b->max_spins, g.st), "forward launch");
      BK(launch_backward(g.wl, b->d_status, b->max_spins, g.st), "backward launch");
      BK(cudaEventRecord(g.done, g.st), "join");
      BK(cudaStreamWaitEvent(s, g.done, 0), "join wait");
    }
    for (auto &g : b->pgroups) BK(cudaStreamWaitEvent(s, g.done, 0), "packed join");
    if (!b->pgroups.empty())  // x += the packed tets' results (the slab tets updated x themselves)
      BK(launch_packed_io(0, b->kind == kSweepMixed, b->d_tets, b->d_iomap, b->total_blocks, b->d_ptrs,
                          nullptr, s),
         "packed update launch");
  }
  return ILU_OK;
}

// One pass of every group on scratch vectors (the tets' scratch and tables
// are real, x and b are a shared scratch buffer: the values are of no use,
// the timing is that of a sweep).  Returns milliseconds, or < 0 on failure.
double time_pass(ilu_batch b, void *scratch) {
  for (int i = 0; i < b->n; ++i) {
    b->h_ptrs[i] = scratch;
    b->h_ptrs[b->n + i] = scratch;
  }
  if (cudaMemcpy(b->d_ptrs, b->h_ptrs, sizeof(void *) * 2 * b->n, cudaMemcpyHostToDevice) != cudaSuccess) return -1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = -1;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, b->cap);
    if (record_passes(b, 1) != ILU_OK) break;
    cudaEventRecord(e1, b->cap);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best < 0 || ms < best)) best = ms;  // the first pass warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaMemcpy(b->h_status, b->d_status, sizeof(LaunchStatus), cudaMemcpyDeviceToHost) != cudaSuccess ||
      b->h_status->code != 0)
    return -1;
  return best;
}

// Autotuner: layers per slab CTA x cluster policy, timed on the batch itself.
ilu_status tune(ilu_batch b) {
  bool slab = false;
  for (const auto &v : b->views) slab = slab || !v.packed;
  if (!slab) return build(b, 0, false);  // packed tets only: nothing to tune
  size_t nmax = 0;
  for (const auto &v : b->views) nmax = std::max(nmax, v.nnodes);
  void *scratch = nullptr;
  BK(cudaMalloc(&scratch, nmax * sizeof(double)), "cudaMalloc tuning scratch");
  BK(cudaMemset(scratch, 0, nmax * sizeof(double)), "cudaMemset tuning scratch");
  int best_zb = 0;
  bool best_largest = false;
  double best_ms = -1;
  for (int zb : {1, 2, 4})
    for (bool largest : {false, true}) {
      free_plan(b);
      if (build(b, zb, largest) != ILU_OK) continue;
      const double ms = time_pass(b, scratch);
      if (ms > 0 && (best_ms < 0 || ms < best_ms)) {
        best_ms = ms;
        best_zb = zb;
        best_largest = largest;
      }
    }
  cudaFree(scratch);
  free_plan(b);
  b->tuned_zb = best_zb;
  b->tuned_largest = best_largest;
  b->tuned_ms = best_ms;
  return build(b, best_zb, best_largest);
}

ilu_status capture(ilu_batch b, int sweeps) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  BK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed), "begin capture");
  ilu_status st = record_passes(b, sweeps);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
  if (st != ILU_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(ILU_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return fail(ILU_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  b->graph_sweeps = sweeps;
  return ILU_OK;
}

}  // namespace

extern "C" {

ilu_status ilu_batch_create(const ilu_tet *tets, int n, const ilu_opts *opts, ilu_batch *out) {
  ilu::DeviceRestore keep_device;
  if (!out) return fail(ILU_EINVAL, "null output handle");
  *out = nullptr;
  if (!tets || n <= 0) return fail(ILU_EINVAL, "empty batch");
  ilu_batch b = new (std::nothrow) ilu_batch_s;
  if (!b) return fail(ILU_ENOMEM, "out of host memory");
  b->n = n;
  b->tets.assign(tets, tets + n);
  b->views.resize(n);
  for (int i = 0; i < n; ++i) {
    if (!tet_view(tets[i], &b->views[i])) {
      delete b;
      return fail(ILU_EINVAL, "tet " + std::to_string(i) + " is null or has no device part");
    }
    const TetView &v = b->views[i];
    if (v.failed) {
      delete b;
      return fail(ILU_EINVAL, "tet " + std::to_string(i) + " failed earlier");
    }
    if (v.device != b->views[0].device || v.precision != b->views[0].precision) {
      delete b;
      return fail(ILU_EINVAL, "the tets of a batch share one device and one precision");
    }
  }
  b->device = b->views[0].device;
  b->precision = b->views[0].precision;
  b->kind = b->views[0].kind;
  if (opts && opts->max_wait_spins > 0) b->max_spins = opts->max_wait_spins;
  if (cudaSetDevice(b->device) != cudaSuccess) {
    delete b;
    return fail(ILU_ECUDA, "cudaSetDevice");
  }
  ilu_status st;
  if (opts && opts->slabs > 0) {
    b->explicit_slabs = opts->slabs;  // an explicit partition, as ilu_opts.slabs for one tet
    st = build(b, 0, false);
  } else {
    st = tune(b);
  }
  if (st != ILU_OK) {
    const std::string msg = ilu_last_error();
    release(b);
    return fail(st, msg);
  }
  *out = b;
  return ILU_OK;
}

ilu_status ilu_batch_destroy(ilu_batch b) {
  ilu::DeviceRestore keep_device;
  if (!b) return ILU_OK;
  release(b);
  return ILU_OK;
}

ilu_status ilu_batch_launches(ilu_batch b, int *per_sweep) {
  if (!b || !per_sweep) return fail(ILU_EINVAL, "null argument");
  int n = 0;
  for (int op = 0; op < 3; ++op) n += b->rblocks[op] > 0;  // the residual, one launch per stencil form
  n += (int)b->pgroups.size() + 2 * (int)b->groups.size() + (b->pgroups.empty() ? 0 : 1);
  *per_sweep = n;
  return ILU_OK;
}

ilu_status ilu_batch_smooth(ilu_batch b, void *const *x, const void *const *bv, int sweeps, void *stream) {
  ilu::DeviceRestore keep_device;
  if (!b || !x || !bv) return fail(ILU_EINVAL, "null argument");
  if (b->failed) return fail(ILU_ECUDA, "batch failed earlier; destroy it");
  if (sweeps < 0) return fail(ILU_EINVAL, "negative sweep count");
  if (sweeps == 0) return ILU_OK;
  for (int i = 0; i < b->n; ++i)
    if (!x[i] || !bv[i]) return fail(ILU_EINVAL, "null vector for tet " + std::to_string(i));
  BK(cudaSetDevice(b->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  // the staging buffer is reused once the previous pointer upload has run
  BK(cudaEventSynchronize(b->ptr_ev), "pointer upload");
  for (int i = 0; i < b->n; ++i) {
    b->h_ptrs[i] = x[i];
    b->h_ptrs[b->n + i] = const_cast<void *>(bv[i]);
  }
  BK(cudaMemcpyAsync(b->d_ptrs, b->h_ptrs, sizeof(void *) * 2 * b->n, cudaMemcpyHostToDevice, st),
     "pointer upload");
  BK(cudaEventRecord(b->ptr_ev, st), "pointer upload");
  if (!b->exec || b->graph_sweeps != sweeps) {
    ilu_status s = capture(b, sweeps);
    if (s != ILU_OK) {
      b->failed = true;
      return s;
    }
  }
  cudaError_t e = cudaGraphLaunch(b->exec, st);
  if (e != cudaSuccess) {
    b->failed = true;
    return fail(ILU_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(b->h_status, b->d_status, sizeof(LaunchStatus), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    b->failed = true;
    return fail(ILU_ECUDA, std::string("batch sweep: ") + cudaGetErrorString(e));
  }
  if (b->h_status->code != 0) {
    b->failed = true;
    return fail(ILU_ETIMEOUT, "a bounded device wait ran out in the batch (slab " +
                                  std::to_string(b->h_status->where) + ", level " +
                                  std::to_string(b->h_status->level) + ")");
  }
  return ILU_OK;
}

}  // extern "C"
