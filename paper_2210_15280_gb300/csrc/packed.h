// packed.h -- the packed substitution kernels of the FP32 sweeps (packed.cu)
// and their host-side row schedules (packed_plan.cpp).
//
// A packed launch gives every macro-tetrahedron one CTA of kPackedLanes
// threads (up to level 7) or one cluster of two CTAs of kPackedClusterLanes
// threads (level 8), which runs the tet's whole forward substitution and then
// its whole backward substitution (Alg. 2 of arXiv 2210.15280) without
// waiting on any other tet.  In a cluster every CTA keeps the whole ring:
// a lane stores each result into its own CTA's ring and into the other's, so
// every producer read is a local shared-memory load.  The interior rows (y, z) are packed onto the cluster's lanes: a
// lane owns one row at a time, keeps that row's surrogate polynomials in
// registers and computes one point of it per step; the cluster meets at a
// barrier every q steps (q, the schedule's quantum: 1, 2 or 4 by level).
//
// The schedule -- which lane owns which row from which step on -- is computed
// on the host once per level (packed_plan.cpp): a list schedule that starts
// each row as soon as its producer rows are far enough ahead and a lane is
// free, with row starts on multiples of the quantum so that the lanes of a
// warp change rows on the same few steps.  The backward substitution runs
// the same schedule backwards in time (step T - 1 - tau of the forward
// pass): every forward dependency, reversed, is a backward one, so the
// reversed schedule is valid, and every row stays on its lane.
//
// Packed layout.  Point (x, y, z) of a row that starts at forward step s on
// lane l has the slot (s + x - 1, l) of a float array of T steps x n lanes
// (n: the cluster's lanes) in four-step blocks: step s of lane l at
// ((s / 4) * n + l) * 4 + s % 4 (packed_index32).  The residual
// writes r there, the forward pass replaces it by its result and the
// backward pass by its own; an update kernel adds the latter to x.  The
// passes move one 16-byte block per lane every four steps, the lanes of a warp
// on consecutive blocks; a row's consecutive points fill whole blocks.
#pragma once
#include <string>
#include <vector>

#if defined(__CUDACC__)
#define ILU_PACKED_HD __host__ __device__
#else
#define ILU_PACKED_HD
#endif

namespace ilu {

constexpr int kPackedLanes = 384;         // threads (row lanes) of a packed CTA on its own
constexpr int kPackedClusterLanes = 320;  // threads of each CTA of a two-CTA cluster (the whole ring of
                                          // both CTAs' lanes fits the shared memory of each)
constexpr int kPackedRing = 32;           // steps of each lane's results kept in shared memory
// words per ring row for a schedule of n lanes: column n is never written
ILU_PACKED_HD constexpr int packed_ring_row(int lanes) { return lanes + 8; }
constexpr int kPackedQueue = 8;    // input queue slots per lane
constexpr int kPackedPre = 7;      // input prefetch distance in steps (below the slot count: the
                                   // entry read at a step is never the one being refilled)
constexpr int kPackedBlock = 8;    // steps per unrolled block of the kernels' loop; T is a multiple
constexpr int kPackedMaxLevel = 8; // highest level the packed kernels take
constexpr int kPackedMaxDegree = 6;  // highest row degree (its coefficients fill the shared memory)

// A producer code tells a consumer row where the values of one of its three
// producer rows are (bits 30-31 the mode): the producer's lane (over the
// whole cluster, at most 1016) in bits 0-9, the step distance k0 of the first value the
// consumer reads at a step (the second is written one step later) in bits
// 10-29, and
//   kProdNone    no such interior row (read from the ring column nothing
//                writes: 0);
//   kProdRing    k0 <= min(kPackedRing - 1, kPackedRing + 1 - q): read from
//                the producer lane's ring;
//   kProdGlobal  further behind: read back from the packed array in global
//                memory, prefetched like the inputs.
enum { kProdNone = 0, kProdRing = 1, kProdGlobal = 2 };
inline int prod_code(int mode, int slot, int k0) { return (mode << 30) | slot | (k0 << 10); }

// One row of a schedule (32 bytes), in the pass's own steps:
//   sw_dlo_far  sw | (lo - sw) << 16 | far << 20: the switch step sw (q - 1
//               mod q), the step lo of the row's first point (lo - sw in
//               1..q), bit j of far set if producer j comes through the queue;
//   nyz         n | y << 10 | z << 20 (n = points of the row);
//   r01, r2rid  R0 | R1 << 15 and R2 | row id << 15: R_j is the word, in
//               the ring (rows of packed_ring_row(lanes) words), of the value
//               read at the first step of the kPackedBlock-step block holding
//               sw (column `lanes`, which nothing writes, if the producer row
//               does not exist or comes through the queue);
//   tt0         the row coordinate t of the point at step sw (float bits);
//   p[3]        the three producer codes.
struct PackedEntry {
  int sw_dlo_far, nyz, r01, r2rid, tt0, p[3];
};

// slot of step s, lane l in the packed array of `lanes` lanes
ILU_PACKED_HD inline int packed_index32(int s, int l, int lanes) { return (((s >> 2) * lanes + l) << 2) + (s & 3); }

struct PackedPlan {
  int N = 0, lanes = 0, q = 1, nsteps = 0;  // lanes: all lanes of the tet's CTA or cluster; q: the start
                                            // quantum; nsteps = T, the steps of either pass (a multiple of
                                            // kPackedBlock)
  std::vector<PackedEntry> fwd, bwd;  // grouped by lane, each lane's rows in step order
  std::vector<int> lane_off;          // lanes + 1 offsets into either list
  std::vector<int> row_map;           // per row id: forward first step | lane << 20
};

// Schedule of a level-L tet (N = 2^L) on `lanes` lanes with row starts on
// multiples of q (1, 2 or 4).  The forward producers of row (y, z) are
// (y-1, z), (y, z-1), (y+1, z-1); the backward ones (y+1, z), (y, z+1),
// (y-1, z+1).  False (with err) if a check of the schedule fails.
bool make_packed_plan(int N, int lanes, int q, PackedPlan *out, std::string *err);
// The start quantum, the cluster size (CTAs per tet) and the lanes of the
// kernels' schedules at N.
int packed_quantum(int N);
int packed_cluster(int N);
int packed_lanes(int N);
// The plan on packed_lanes(N) lanes with the level's quantum, computed once
// per level and kept for the life of the process; null (with err) if the
// schedule fails.
const PackedPlan *packed_plan_cached(int N, std::string *err);

}  // namespace ilu
