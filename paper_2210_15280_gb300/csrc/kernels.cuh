// kernels.cuh -- device-side data of one macro-tetrahedron and the launchers
// of the sweep kernels (arXiv 2210.15280, Alg. 2 with the V2 boundary rule).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "grid.h"

struct ilu_tet_s;

namespace ilu {

// Partition of a tet for one substitution: zb face layers per z-slab (CTA),
// wpl compute warps per layer, P slabs launched as clusters of csize CTAs;
// prog = first progress word of the slabs in the flag array, ticket = the
// ticket counter of the clusters.
struct WaveGeom {
  int zb, wpl, P, csize, prog, ticket;
};

// Band layout of the FP32 sweeps (band.cu): per band (z,k), index
// (z-1) * (band_kmax(N)+1) + k, the offset of its [step-1][32] block in the
// band array, of its edge stream and of the stream to the next CTA (or -1).
struct BandInfo {
  int64_t off, hoff, voff;
};

struct BandDev {
  const BandInfo *info;
  const int *cta;     // CTAs in dependency order: group << 16 | band
  const int *tiles;   // residual/update tiles: z << 20 | k << 14 | chunk
  void *w;            // band array (float)
  unsigned long long *streams;  // tagged words exchanged between CTAs
  int *epoch;         // launch tag counter (bumped by the first tile kernel of a sweep)
  int ncta, ntiles, Z;
};

// Row schedules of the packed substitutions (packed.h): the PackedEntry
// records (two int4 each) of either pass grouped by lane, the lane offsets
// (the same for both), per row id its forward first step | lane << 20, the
// packed step-major array [nsteps][lanes] and its step count.
struct PackedDev {
  const int4 *ent_f, *ent_b;
  const int *off;
  const int *row_map;
  float *pw;
  int nsteps;
  int lanes;  // lanes of the schedule: all lanes of the tet's CTA or cluster
};

// Everything a kernel needs to know about one tet.  Plain old data so that it
// can live in a device array for batched launches.
struct DevTet {
  int L, N;
  double h;
  int dx;          // surrogate degree in x = row polynomial degree
  int rstride;     // coefficients per function in the row tables (4, 8 or 16, zero padded)
  WaveGeom fwd, bwd;
  int const_kappa;
  const void *tabF;  // rows x 7 x rstride (float or double)
  const void *tabB;  // rows x 8 x rstride
  const double *kappa;  // kappa at every grid point (variable coefficient)
  void *w;           // scratch, full grid, element type of the sweep
  int *flags;        // progress words of the slabs and the two ticket counters
  double A15[15];    // constant stencil
  double Wstar[100]; // edge-star weights (variable coefficient)
  BandDev band;      // FP32 band sweeps (null info when not used)
  PackedDev pk;      // packed substitution schedules (null when not used)
  const void *pkF;   // packed kernels' FP32 row polynomials: [row][k = 0..dx][4 function pairs] float2,
  const void *pkB;   // forward and backward (null when not used)
  const int *chunks; // residual work list: first point x | y << 10 | z << 20 of each run of 32
                     // interior points in lexicographic order (chunk_point in grid.h)
  int nchunks;
  const int *strips; // constant-stencil residual work list: x0 | y0 << 10 | z << 20 of each strip
                     // (residual_strip_list)
  int nstrips;
  const void *astore;    // variable kappa, stored operator: coefficient of direction d (d != centre) of
                         // row p at astore[(d < 7 ? d : d - 1) * astride + p], double (float in F32
                         // sweeps); null: assembled on the fly
  int64_t astride;
  const void *bnd;       // boundary variant V1: 8 values per cell-boundary point (sweep precision): its exact
                         // L^p_d (d in D_l) and 1/D^p; or null
  const int *bnd_off;    // its row offsets (bnd_record in grid.h)
  const double *valsF;   // FP64 sweeps with tabulated surrogate values, 8 per grid point at 8 * index:
  const double *valsB;   // forward L~^p_d (d in D_l) and 0; backward 1/D~^p, L~^{p-d}_d.  Null: the
                         // substitutions evaluate the row polynomials themselves
};

struct LaunchStatus {
  int code;     // 0 ok, otherwise an ilu_status value
  int where;    // slab that gave up
  int level;    // level it was waiting for
  int pad;
};

// precision of the sweep: W = element type of w and the row tables,
// X = element type of x and b, R = type the residual is computed in
enum SweepKind { kSweepF64 = 0, kSweepF32 = 1, kSweepMixed = 2 };

// packed: write r into the tet's packed array (t.pk) instead of r_out.  The
// grid holds as many CTAs as the GPU keeps resident at once (at most
// nblocks_cap); *nblocks_used receives it, the number of partial norms
// written to `partials`.
cudaError_t launch_residual(const DevTet &t, int kind, const void *x, const void *b, void *r_out, double *partials,
                            int nblocks_cap, int *nblocks_used, cudaStream_t st, bool packed = false);
// How a tet's residual gets its operator: the constant stencil, assembled on
// the fly from kappa at the grid points, or the stored coefficients.
constexpr int kOpConst = 0, kOpStar = 1, kOpStored = 2;
inline int residual_op(const DevTet &t) { return t.const_kappa ? kOpConst : (t.astore ? kOpStored : kOpStar); }
// Residual of many tets with the same residual_op in one launch: block i of
// the 1-D grid is block bmap[i].y of tet bmap[i].x (residual_blocks(N) per
// tet, residual_strip_blocks(N) for the constant stencil); tets, bmap and the per-tet pointer arrays (indexed by tet) are device
// memory.  Writes w of each tet, or its packed array if it has one; no norms.
cudaError_t launch_residual_batch(const DevTet *tets, const int2 *bmap, int total_blocks, int kind, int op,
                                  const void *const *xs, const void *const *bs, cudaStream_t st);
cudaError_t launch_norm_finish(const double *partials, int n, double *out, cudaStream_t st);
// assemble the 14 off-diagonal coefficients of every interior row (variable
// kappa) into A (14 planes of t.astride doubles), the values the on-the-fly
// residual computes
cudaError_t launch_stencil_store(const DevTet &t, void *A, bool f32, cudaStream_t st);

// Clusters of a substitution launch handed out as tickets: tets in `order`,
// tet order[j] taking tickets [prefix[j], prefix[j+1]) in dependency order.
// `ticket` is the zeroed counter; the backward launch adds x (per tet in xs,
// or x0 for every tet).  All pointers are device memory.
struct BatchMap {
  const int *prefix;
  const int *order;
  int n;
  int *ticket;
  void *const *xs;
  void *x0;
};

// One substitution launch over one or more tets (same sweep kind and row
// polynomial layout): block sizes, shared memory and cluster shapes are the
// maxima over its tets.
struct WaveLaunch {
  const DevTet *tets;  // device array
  int kind;            // SweepKind
  int reg;             // register path: row degree (0..7); -1: rows read from shared memory;
                       // kWaveTabulated: surrogate values read from the tet's tables
  int dxp;             // padded coefficients per row function (rstride of the tets)
  BatchMap map_f, map_b;
  int block_f, block_b;    // threads per CTA
  size_t smem_f, smem_b;   // dynamic shared memory per CTA
  int csize_f, csize_b;    // CTAs per cluster
  int clusters_f, clusters_b;
  int maxP_f, maxP_b;      // most slabs of any tet
  bool v1;                 // some tet uses boundary variant V1 (its stored factors are consulted)
};

// Cluster sizes the launchers consider, largest first.
constexpr int kClusterCands = 6;
constexpr int kClusterSizes[kClusterCands] = {16, 12, 8, 4, 2, 1};
// With cluster_query (int[1 + kClusterCands]) set nothing is launched:
// [0] receives the largest cluster size the device can schedule for the
// launch's shape, [1 + i] how many clusters of min(kClusterSizes[i], maxP)
// CTAs can be resident at once (0 if none fit).
cudaError_t launch_forward(const WaveLaunch &L, LaunchStatus *status, long long max_spins, cudaStream_t st,
                           int *cluster_query = nullptr);
cudaError_t launch_backward(const WaveLaunch &L, LaunchStatus *status, long long max_spins, cudaStream_t st,
                            int *cluster_query = nullptr);
// reg: the WaveLaunch.reg code of the launch
size_t wave_smem_bytes(int N, const WaveGeom &g, int kind, int dxp, int reg, bool forward);
// FP32/MIXED sweeps of degree <= 7 keep each row's polynomials in registers
// (CTAs of at most 16 warps); otherwise they are read from shared memory.
bool wave_uses_registers(int kind, int dx);
// WaveLaunch.reg value of FP64 sweeps that read tabulated surrogate values
constexpr int kWaveTabulated = -2;
// Highest level whose tabulated-value staging fits a CTA's shared memory.
constexpr int kTabulatedMaxLevel = 9;
// Fill valsF / valsB (8 doubles per grid point each) from the FP64 row
// tables of t, with the arithmetic of the substitutions' own evaluation.
cudaError_t launch_tabulate(const DevTet &t, double *valsF, double *valsB, cudaStream_t st);
constexpr int kResidualCPW = 4;  // consecutive 32-point chunks per warp of the residual launches
int residual_blocks(int N);  // blocks of the residual launch (8 warps of kResidualCPW row chunks each)
int rowgrid_blocks(int N);   // blocks of the row-per-warp reductions (interior norm)
int residual_chunks(int N);
void residual_chunk_list(int N, int *out);
// Strips of the constant-stencil residual: a warp takes the interior points
// (x0 .. x0 + kStripWidth - 1, y, z) of kStripRows consecutive rows y0 ..;
// z-major, then x0, then y0.
constexpr int kStripWidth = 30, kStripRows = 16;
int residual_strips(int N);
void residual_strip_list(int N, int *out);
int residual_strip_blocks(int N);  // blocks of 8 warps, a strip per warp

// ---- FP32 band sweeps (band.cu)

// One forward or backward band launch over one or more tets: tickets map to
// (tet, CTA) through map.prefix (CTAs per tet) and map.order.
struct BandLaunch {
  const DevTet *tets;
  BatchMap map_f, map_b;
  int ctas;  // total CTAs
  int Z;     // warps (layers) per CTA, 1..8
  int reg;   // row degree held in registers, 0..7 (rstride 4 for <= 3, else 8)
  bool v1;   // some tet uses boundary variant V1 (its stored factors are consulted)
};
size_t band_smem_bytes(int Z);
cudaError_t launch_band_sub(bool forward, const BandLaunch &L, LaunchStatus *status, long long max_spins,
                            cudaStream_t st);
// tiles of all tets (tet i owns tiles [tprefix[i], tprefix[i+1])): mode 0
// r = b - A x into the band array (with per-tile ||r||^2 in partials, may be
// null), mode 1 copy of x into the band array.  xs/bs: device arrays of
// per-tet pointers, or null and x1/b1 for a single tet.
cudaError_t launch_band_in(int kind, int mode, const DevTet *tets, const int *tprefix, int ntets, int total_tiles,
                           const void *const *xs, const void *const *bs, const void *x1, const void *b1,
                           double *partials, cudaStream_t st);
// x += band array (per tet)
cudaError_t launch_band_update(int kind, const DevTet *tets, const int *tprefix, int ntets, int total_tiles,
                               void *const *xs, void *x1, cudaStream_t st);

// ---- packed substitutions (packed.cu): one CTA per tet (level 8: a cluster
// of two) runs its forward and backward substitution on the tet's packed array (which holds r on entry and
// the backward result on exit).  reg: the degree of the packed row tables (3
// or 6); v1: some tet uses boundary variant V1.  order (device, nullable): the
// tet of each CTA (cluster).
struct PackedLaunch {
  const DevTet *tets;
  const int *order;
  int ntets;
  int reg;  // degree of the row tables (3 or 6)
  int q;    // the schedules' start quantum (1, 2 or 4; the same for every tet of the launch)
  int cl;   // CTAs per tet (1 or 2; the same for every tet of the launch)
  bool v1;
  // launched as a programmatic dependent of the stream's previous kernel
  // (itself a packed launch): its CTAs are dispatched once every CTA of that
  // launch has started, and never wait for its results.  The caller joins
  // both launches to whatever follows them with events.
  bool after_packed;
};
size_t packed_smem_bytes(int reg, int cl);
cudaError_t launch_packed(const PackedLaunch &L, cudaStream_t st);
// Between a tet's lexicographic vectors and its packed array, over the
// residual chunk list (block i of the grid is block bmap[i].y of tet
// bmap[i].x, or block i of tets[0] when bmap is null): mode 0 adds the packed
// values to x (per tet in xs, or x1), mode 1 copies the interior of x (a
// vector, converted to float) into the packed array.  Tets without a packed
// array are skipped.  f64: x is double, else float.
cudaError_t launch_packed_io(int mode, bool f64, const DevTet *tets, const int2 *bmap, int total_blocks,
                             void *const *xs, void *x1, cudaStream_t st);

// ---- host-side views shared by the entry-point files (capi.cu defines them)

// what a batch needs to know of a tet handle
struct TetView {
  const DevTet *dev;  // host copy of the device descriptor
  int N, dx, rstride, device, precision, kind;
  int reg;  // WaveLaunch.reg code of its substitutions
  size_t nnodes;
  bool failed;
  bool packed;  // its substitutions run on the packed kernels (cost: steps of both passes)
  int packed_steps;
  int packed_q;  // their schedules' start quantum
  int packed_cl; // and CTAs per tet
};
bool tet_view(ilu_tet_s *t, TetView *v);
// partition of one substitution (requested > 0: about that many slabs)
WaveGeom wave_geom(int N, int kind, int dxp, int reg, bool fwd, int requested);

// solver helpers on full-grid vectors (double if f64, else float)
constexpr int kDotPartials = 512;
cudaError_t launch_dot(bool f64, const void *a, const void *b, long long n, double *partials, double *out,
                       cudaStream_t st);
cudaError_t launch_axpy(bool f64, void *y, const void *x, double a, long long n, cudaStream_t st);
cudaError_t launch_xpay(bool f64, void *p, const void *z, double b, long long n, cudaStream_t st);
cudaError_t launch_copy(bool src_f64, bool dst_f64, const void *src, void *dst, long long n, cudaStream_t st);
cudaError_t launch_interior_norm(int N, bool f64, const void *v, double *partials, int cap, double *out,
                                 cudaStream_t st);

}  // namespace ilu
