// capi.cu -- the extern "C" entry points declared in include/ilu.h.
//
// A handle (ilu_tet) owns the FP64 host set-up (setup.cpp) and its device
// part: the per-row surrogate tables in the sweep precision, kappa at the grid
// points for a variable coefficient, one full-grid scratch vector w (the
// residual, then the substitution result, in place), the slab progress flags
// and a status word that bounded device waits write on timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ilu.h"
#include "hooks.h"
#include "kernels.cuh"
#include "packed.h"
#include "setup.h"

using namespace ilu;

namespace {

thread_local std::string g_err;

ilu_status fail(ilu_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

ilu_status cuda_fail(cudaError_t e, const char *what) {
  return fail(ILU_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

constexpr long long kDefaultSpins = 4000000;  // ~a few seconds of polling with nanosleep

}  // namespace

struct ilu_tet_s {
  HostTet host;
  int precision = ILU_MIXED;
  int device = -1;
  long long max_spins = kDefaultSpins;
  bool failed = false;
  DevTet dev = {};
  int nflags = 0;
  void *d_tabF = nullptr, *d_tabB = nullptr, *d_w = nullptr;
  double *d_kappa = nullptr, *d_partials = nullptr, *d_norms = nullptr;
  int *d_flags = nullptr;
  DevTet *d_dev = nullptr;  // device copy of dev
  // FP32 band sweeps (band.cu): layout tables, band array, streams
  bool use_band = false;
  int requested_slabs = 0, kernel_choice = ILU_KERNEL_AUTO, stencil_choice = ILU_STENCIL_AUTO;
  int perm[4] = {0, 1, 2, 3};  // vertex order used (ILU_ORIENT_LFA)
  int max_cluster = 0;         // cap on CTAs per cluster (0: none)
  void *d_astore = nullptr;  // stored off-diagonal coefficients, 14 planes of nnodes (variable kappa; float in F32)
  void *d_bnd = nullptr;       // boundary variant V1: exact factor records (sweep precision)
  int *d_bnd_off = nullptr;    // and their row offsets
  bool tabulate = false;       // FP64 substitutions read tabulated surrogate values
  double *d_valsF = nullptr, *d_valsB = nullptr;  // those tables (8 doubles per grid point each)
  int band_Z = 8, band_ntiles = 0, band_ncta = 0;
  BandInfo *d_binfo = nullptr;
  int *d_bint = nullptr;  // CTA list, tile list, cluster map {0, ncta, 0}, tile prefix {0, ntiles}, epoch
  void *d_bw = nullptr;
  unsigned long long *d_bstreams = nullptr;
  BandLaunch bl = {};
  // packed substitutions (packed.cu): schedules of both directions
  bool use_packed = false;
  void *d_pkF = nullptr, *d_pkB = nullptr;  // compact row polynomials of the packed kernels
  int4 *d_pk = nullptr;      // schedules, lane offsets and row map in one block
  float *d_pkw = nullptr;    // the packed array [T][lanes]
  PackedLaunch pl = {};
  const int *band_tprefix = nullptr;
  int *d_map = nullptr;     // cluster prefixes {0, Qf}, {0, Qb} and the order {0}
  int *d_chunks = nullptr;  // residual work list (32-point row chunks)
  int *d_strips = nullptr;  // constant-stencil residual work list (strips)
  WaveLaunch wl = {};       // the forward/backward launch shape of this tet
  LaunchStatus *d_status = nullptr, *h_status = nullptr;
  int nblocks = 0, norms_cap = 0;
  void *d_xs = nullptr, *d_bs = nullptr;  // staging for ilu_smooth_host
  void *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_q = nullptr, *d_zero = nullptr;  // Krylov vectors
  double *d_dot = nullptr, *d_scal = nullptr;  // dot partials, scalars
  double *h_scal = nullptr;                    // pinned copy of the scalars
  // tracing: CUDA event pairs around each kernel launch
  bool prof = false;
  struct Ev {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Ev> ev_used;
  std::vector<cudaEvent_t> ev_pool;
  long long launches = 0;
  std::mutex mu;
  size_t elem() const { return precision == ILU_F32 ? sizeof(float) : sizeof(double); }
  int kind() const { return precision == ILU_F64 ? kSweepF64 : (precision == ILU_F32 ? kSweepF32 : kSweepMixed); }
  // WaveLaunch.reg code of the slab substitutions
  int wave_reg() const {
    if (tabulate) return kWaveTabulated;
    return wave_uses_registers(kind(), host.dx) ? host.dx : -1;
  }
  size_t nnodes() const { return (size_t)grid_nodes(host.N); }
};

namespace {

void free_device(ilu_tet t) {
  if (t->device < 0) return;
  cudaSetDevice(t->device);
  for (auto &e : t->ev_used) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  for (auto e : t->ev_pool) cudaEventDestroy(e);
  t->ev_used.clear();
  t->ev_pool.clear();
  cudaFree(t->d_tabF); cudaFree(t->d_tabB); cudaFree(t->d_w); cudaFree(t->d_kappa); cudaFree(t->d_astore);
  cudaFree(t->d_bnd); cudaFree(t->d_bnd_off);
  cudaFree(t->d_pk); cudaFree(t->d_pkw); cudaFree(t->d_pkF); cudaFree(t->d_pkB);
  t->d_pk = nullptr;
  t->d_pkw = nullptr;
  t->d_pkF = t->d_pkB = nullptr;
  cudaFree(t->d_valsF); cudaFree(t->d_valsB);
  t->d_valsF = t->d_valsB = nullptr;
  t->d_astore = nullptr;
  t->d_bnd = nullptr;
  t->d_bnd_off = nullptr;
  cudaFree(t->d_partials); cudaFree(t->d_norms); cudaFree(t->d_flags); cudaFree(t->d_status);
  cudaFree(t->d_dev); cudaFree(t->d_map); cudaFree(t->d_chunks); cudaFree(t->d_strips);
  t->d_dev = nullptr; t->d_map = nullptr; t->d_chunks = nullptr; t->d_strips = nullptr;
  cudaFree(t->d_binfo); cudaFree(t->d_bint); cudaFree(t->d_bw); cudaFree(t->d_bstreams);
  t->d_binfo = nullptr; t->d_bint = nullptr; t->d_bw = nullptr; t->d_bstreams = nullptr;
  cudaFree(t->d_xs); cudaFree(t->d_bs);
  cudaFree(t->d_r); cudaFree(t->d_z); cudaFree(t->d_p); cudaFree(t->d_q); cudaFree(t->d_zero);
  cudaFree(t->d_dot); cudaFree(t->d_scal);
  if (t->h_scal) cudaFreeHost(t->h_scal);
  t->d_r = t->d_z = t->d_p = t->d_q = t->d_zero = nullptr;
  t->d_dot = t->d_scal = t->h_scal = nullptr;
  if (t->h_status) cudaFreeHost(t->h_status);
  t->d_tabF = t->d_tabB = t->d_w = nullptr;
  t->d_kappa = t->d_partials = t->d_norms = nullptr;
  t->d_flags = nullptr; t->d_status = nullptr; t->h_status = nullptr; t->d_xs = t->d_bs = nullptr;
}

// Partition for one substitution: wpl warps per face layer (one chunk of 32
// rows each at the widest level), as many layers per slab as fit 31 compute
// warps and ~200 KB of shared memory (ring, prefetch slots, row cache).
// Thin slabs are the default: inside a cluster a hop between slabs costs a
// few hundred cycles, while every extra layer adds its warps' issue time to
// each level of the slab.
WaveGeom pick_geom(int N, int kind, int dxp, int reg, bool fwd, int requested) {
  const int layers = std::max(1, N - 3);
  WaveGeom g = {};
  g.wpl = std::max(1, std::min(8, (N / 2 + 31) / 32));
  const int max_warps = reg >= 0 ? 15 : 31;  // plus the communication warp
  int zb = std::max(1, max_warps / g.wpl);
  zb = std::min(zb, requested > 0 ? (layers + requested - 1) / requested : 2);
  zb = std::min(zb, layers);
  while (zb > 1) {
    g.zb = zb;
    if (wave_smem_bytes(N, g, kind, dxp, reg, fwd) <= 200 * 1024) break;
    --zb;
  }
  g.zb = zb;
  g.P = (layers + zb - 1) / zb;
  return g;
}

void choose_geometry(ilu_tet t, int requested) {
  const int N = t->host.N;
  DevTet &d = t->dev;
  d.fwd = pick_geom(N, t->kind(), t->host.rstride, t->wave_reg(), true, requested);
  d.bwd = pick_geom(N, t->kind(), t->host.rstride, t->wave_reg(), false, requested);
  d.fwd.prog = 0;
  d.bwd.prog = d.fwd.P;
  d.fwd.ticket = d.fwd.P + d.bwd.P;
  d.bwd.ticket = d.fwd.ticket + 1;
  t->nflags = d.fwd.P + d.bwd.P + 2;
}

// Launch shape of one tet's substitutions; cluster sizes from the device's
// limit for that shape (one cluster holds the whole tet when it has at most
// that many slabs), then the device copies of the tet and its cluster map.
ilu_status choose_clusters(ilu_tet t) {
  DevTet &d = t->dev;
  const HostTet &h = t->host;
  WaveLaunch &L = t->wl;
  L = {};
  L.tets = t->d_dev;
  L.kind = t->kind();
  L.reg = t->wave_reg();
  L.dxp = h.rstride;
  L.v1 = h.boundary == ILU_BOUNDARY_V1;
  L.block_f = (d.fwd.zb * d.fwd.wpl + 1) * 32;
  L.block_b = (d.bwd.zb * d.bwd.wpl + 1) * 32;
  L.smem_f = wave_smem_bytes(h.N, d.fwd, L.kind, h.rstride, L.reg, true);
  L.smem_b = wave_smem_bytes(h.N, d.bwd, L.kind, h.rstride, L.reg, false);
  L.maxP_f = d.fwd.P;
  L.maxP_b = d.bwd.P;
  int qf[1 + kClusterCands] = {}, qb[1 + kClusterCands] = {};
  CK(launch_forward(L, nullptr, 0, nullptr, qf), "cluster query");
  CK(launch_backward(L, nullptr, 0, nullptr, qb), "cluster query");
  int cf = qf[0], cb = qb[0];
  if (t->max_cluster > 0) {
    cf = std::max(1, std::min(cf, t->max_cluster));
    cb = std::max(1, std::min(cb, t->max_cluster));
  }
  // as few clusters as the limit allows, as evenly filled as possible
  d.fwd.csize = (d.fwd.P + (d.fwd.P + cf - 1) / cf - 1) / ((d.fwd.P + cf - 1) / cf);
  d.bwd.csize = (d.bwd.P + (d.bwd.P + cb - 1) / cb - 1) / ((d.bwd.P + cb - 1) / cb);
  L.csize_f = d.fwd.csize;
  L.csize_b = d.bwd.csize;
  L.clusters_f = (d.fwd.P + L.csize_f - 1) / L.csize_f;
  L.clusters_b = (d.bwd.P + L.csize_b - 1) / L.csize_b;
  const int map[5] = {0, L.clusters_f, 0, L.clusters_b, 0};
  CK(cudaMemcpy(t->d_map, map, sizeof(map), cudaMemcpyHostToDevice), "upload cluster map");
  CK(cudaMemcpy(t->d_dev, &d, sizeof(DevTet), cudaMemcpyHostToDevice), "upload tet");
  L.map_f = {t->d_map, t->d_map + 4, 1, t->d_flags + d.fwd.ticket, nullptr, nullptr};
  L.map_b = {t->d_map + 2, t->d_map + 4, 1, t->d_flags + d.bwd.ticket, nullptr, nullptr};
  return ILU_OK;
}

// Band layout of the FP32 sweeps: offsets of every band's block, edge
// stream and (at the top layer of a CTA's stack) stream to the next CTA;
// the CTA list in dependency order and the residual/update tiles.
struct BandPlan {
  std::vector<BandInfo> info;
  std::vector<int> cta, tiles;
  int64_t wfloats = 0, swords = 0;
};

BandPlan make_band_plan(int N, int Z) {
  BandPlan p;
  const int KB = band_kmax(N) + 1;
  p.info.assign((size_t)std::max(N - 3, 0) * KB, BandInfo{-1, -1, -1});
  for (int z = 1; z <= N - 3; ++z)
    for (int k = band_kmin(z); k < KB; ++k) {
      const int shi = band_shi(N, z, k);
      BandInfo &b = p.info[(size_t)(z - 1) * KB + k];
      b.off = p.wfloats;
      p.wfloats += (int64_t)shi * 32;
      b.hoff = p.swords;  // 16-byte records 0 .. shi + 127
      p.swords += 2 * ((int64_t)shi + 128);
      if (z % Z == 0 && band_exists(N, z + 1, k)) {
        b.voff = p.swords;  // [step 0 .. shi][32]
        p.swords += ((int64_t)shi + 2) * 32;
      }
      for (int ch = 0; ch < (shi + 31) / 32; ++ch) p.tiles.push_back(z << 20 | k << 14 | ch);
    }
  for (int g = 0; 1 + g * Z <= N - 3; ++g)
    for (int k = band_kmin(1 + g * Z); k < KB; ++k) p.cta.push_back(g << 16 | k);
  return p;
}

ilu_status upload_band(ilu_tet t, int requested_slabs) {
  const int N = t->host.N;
  const int layers = std::max(1, N - 3);
  int Z = 8;
  if (requested_slabs > 0) Z = std::min(8, std::max(1, (layers + requested_slabs - 1) / requested_slabs));
  BandPlan p = make_band_plan(N, Z);
  t->band_Z = Z;
  t->band_ncta = (int)p.cta.size();
  t->band_ntiles = (int)p.tiles.size();
  const size_t ni = p.cta.size() + p.tiles.size() + 3 + 2 + 1;
  std::vector<int> ints;
  ints.reserve(ni);
  ints.insert(ints.end(), p.cta.begin(), p.cta.end());
  ints.insert(ints.end(), p.tiles.begin(), p.tiles.end());
  const size_t at_map = ints.size();
  ints.push_back(0); ints.push_back(t->band_ncta); ints.push_back(0);  // CTA prefix {0, ncta}, order {0}
  const size_t at_tp = ints.size();
  ints.push_back(0); ints.push_back(t->band_ntiles);  // tile prefix
  const size_t at_epoch = ints.size();
  ints.push_back(0);
  CK(cudaMalloc(&t->d_binfo, sizeof(BandInfo) * std::max<size_t>(p.info.size(), 1)), "cudaMalloc band tables");
  if (!p.info.empty())
    CK(cudaMemcpy(t->d_binfo, p.info.data(), sizeof(BandInfo) * p.info.size(), cudaMemcpyHostToDevice), "upload band tables");
  CK(cudaMalloc(&t->d_bint, sizeof(int) * ints.size()), "cudaMalloc band tables");
  CK(cudaMemcpy(t->d_bint, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice), "upload band tables");
  CK(cudaMalloc(&t->d_bw, sizeof(float) * std::max<int64_t>(p.wfloats, 1)), "cudaMalloc band array");
  CK(cudaMemset(t->d_bw, 0, sizeof(float) * std::max<int64_t>(p.wfloats, 1)), "cudaMemset band array");
  CK(cudaMalloc(&t->d_bstreams, sizeof(unsigned long long) * std::max<int64_t>(p.swords, 2)), "cudaMalloc streams");
  CK(cudaMemset(t->d_bstreams, 0, sizeof(unsigned long long) * std::max<int64_t>(p.swords, 2)), "cudaMemset streams");
  BandDev &b = t->dev.band;
  b.info = t->d_binfo;
  b.cta = t->d_bint;
  b.tiles = t->d_bint + p.cta.size();
  b.w = t->d_bw;
  b.streams = t->d_bstreams;
  b.epoch = t->d_bint + at_epoch;
  b.ncta = t->band_ncta;
  b.ntiles = t->band_ntiles;
  b.Z = Z;
  t->nblocks = std::max(t->nblocks, t->band_ntiles);
  BandLaunch &L = t->bl;
  L.tets = t->d_dev;
  L.ctas = t->band_ncta;
  L.Z = Z;
  L.reg = t->host.dx;
  L.v1 = t->host.boundary == ILU_BOUNDARY_V1;
  L.map_f = {t->d_bint + at_map, t->d_bint + at_map + 2, 1, t->d_flags + t->dev.fwd.ticket, nullptr, nullptr};
  L.map_b = {t->d_bint + at_map, t->d_bint + at_map + 2, 1, t->d_flags + t->dev.bwd.ticket, nullptr, nullptr};
  t->band_tprefix = t->d_bint + at_tp;
  return ILU_OK;
}

// The FP32 row tables ([row][pair p][k][2], k padded to rstride) rearranged
// for the packed kernels: [row][k][pair p][2], 32 bytes per k, with
// packed_degree(dx) + 1 coefficients (zero padded), the degree the kernels
// are instantiated for: every tet of a row-table class shares one launch.
int packed_degree(int dx) { return dx <= 3 ? 3 : kPackedMaxDegree; }
void compact_rows(const HostTet &h, const std::vector<float> &tab, std::vector<float> &out) {
  const int64_t R = num_rows(h.N);
  const int S = h.rstride, K = packed_degree(h.dx) + 1;
  out.assign((size_t)R * K * 8, 0.0f);
  for (int64_t r = 0; r < R; ++r)
    for (int k = 0; k < K; ++k)
      for (int p = 0; p < 4; ++p)
        for (int j = 0; j < 2; ++j)
          out[(((size_t)r * K + k) * 4 + p) * 2 + j] = k < S ? tab[(((size_t)r * 4 + p) * S + k) * 2 + j] : 0.0f;
}

ilu_status upload_packed_tables(ilu_tet t) {
  const HostTet &h = t->host;
  std::vector<float> cf, cb;
  compact_rows(h, h.tabF32, cf);
  compact_rows(h, h.tabB32, cb);
  if (!t->d_pkF) CK(cudaMalloc(&t->d_pkF, sizeof(float) * std::max<size_t>(cf.size(), 4)), "cudaMalloc packed tables");
  if (!t->d_pkB) CK(cudaMalloc(&t->d_pkB, sizeof(float) * std::max<size_t>(cb.size(), 4)), "cudaMalloc packed tables");
  if (!cf.empty()) CK(cudaMemcpy(t->d_pkF, cf.data(), sizeof(float) * cf.size(), cudaMemcpyHostToDevice), "upload packed tables");
  if (!cb.empty()) CK(cudaMemcpy(t->d_pkB, cb.data(), sizeof(float) * cb.size(), cudaMemcpyHostToDevice), "upload packed tables");
  t->dev.pkF = t->d_pkF;
  t->dev.pkB = t->d_pkB;
  return ILU_OK;
}

ilu_status upload_packed(ilu_tet t) {
  {
    ilu_status ts = upload_packed_tables(t);
    if (ts != ILU_OK) return ts;
  }
  const int N = t->host.N;
  std::string err;
  const PackedPlan *pl = packed_plan_cached(N, &err);
  if (!pl) return fail(ILU_EINVAL, err);
  const size_t ne = pl->fwd.size();
  const int lanes = pl->lanes;
  static_assert(sizeof(PackedEntry) == 2 * sizeof(int4), "a schedule entry is two int4");
  // one block: forward entries, backward entries, lane offsets, row map
  const size_t ints = 16 * ne + (lanes + 1) + pl->row_map.size();
  std::vector<int> blob(std::max<size_t>(ints, 4), 0);
  if (ne) {
    std::memcpy(blob.data(), pl->fwd.data(), sizeof(PackedEntry) * ne);
    std::memcpy(blob.data() + 8 * ne, pl->bwd.data(), sizeof(PackedEntry) * ne);
  }
  std::memcpy(blob.data() + 16 * ne, pl->lane_off.data(), sizeof(int) * (lanes + 1));
  if (!pl->row_map.empty())
    std::memcpy(blob.data() + 16 * ne + lanes + 1, pl->row_map.data(), sizeof(int) * pl->row_map.size());
  CK(cudaMalloc(&t->d_pk, sizeof(int) * blob.size()), "cudaMalloc packed schedule");
  CK(cudaMemcpy(t->d_pk, blob.data(), sizeof(int) * blob.size(), cudaMemcpyHostToDevice), "upload packed schedule");
  CK(cudaMalloc(&t->d_pkw, sizeof(float) * (size_t)pl->nsteps * lanes), "cudaMalloc packed array");
  CK(cudaMemset(t->d_pkw, 0, sizeof(float) * (size_t)pl->nsteps * lanes), "cudaMemset packed array");
  const int *base = reinterpret_cast<const int *>(t->d_pk);
  PackedDev &p = t->dev.pk;
  p.ent_f = t->d_pk;
  p.ent_b = t->d_pk + 2 * ne;
  p.off = base + 16 * ne;
  p.row_map = base + 16 * ne + lanes + 1;
  p.pw = t->d_pkw;
  p.nsteps = pl->nsteps;
  p.lanes = pl->lanes;
  PackedLaunch &L = t->pl;
  L.tets = t->d_dev;
  L.order = nullptr;
  L.ntets = 1;
  L.reg = packed_degree(t->host.dx);
  L.q = pl->q;
  L.cl = pl->lanes > kPackedLanes ? 2 : 1;
  L.v1 = t->host.boundary == ILU_BOUNDARY_V1;
  return ILU_OK;
}

ilu_status upload(ilu_tet t) {
  HostTet &h = t->host;
  CK(cudaSetDevice(t->device), "cudaSetDevice");
  const size_t nn = t->nnodes();
  const bool f64 = t->precision == ILU_F64;
  const size_t nf = f64 ? h.tabF64.size() : h.tabF32.size(), nb = f64 ? h.tabB64.size() : h.tabB32.size();
  const size_t es = f64 ? sizeof(double) : sizeof(float);
  CK(cudaMalloc(&t->d_tabF, std::max<size_t>(nf, 1) * es), "cudaMalloc tables");
  CK(cudaMalloc(&t->d_tabB, std::max<size_t>(nb, 1) * es), "cudaMalloc tables");
  if (nf) CK(cudaMemcpy(t->d_tabF, f64 ? (const void *)h.tabF64.data() : (const void *)h.tabF32.data(), nf * es,
                        cudaMemcpyHostToDevice), "upload tables");
  if (nb) CK(cudaMemcpy(t->d_tabB, f64 ? (const void *)h.tabB64.data() : (const void *)h.tabB32.data(), nb * es,
                        cudaMemcpyHostToDevice), "upload tables");
  if (!h.const_kappa) {
    CK(cudaMalloc(&t->d_kappa, nn * sizeof(double)), "cudaMalloc kappa");
    CK(cudaMemcpy(t->d_kappa, h.kappa.data(), nn * sizeof(double), cudaMemcpyHostToDevice), "upload kappa");
  }
  CK(cudaMalloc(&t->d_w, nn * t->elem()), "cudaMalloc scratch");
  CK(cudaMemset(t->d_w, 0, nn * t->elem()), "cudaMemset scratch");
  CK(cudaMalloc(&t->d_flags, sizeof(int) * t->nflags), "cudaMalloc flags");
  CK(cudaMemset(t->d_flags, 0, sizeof(int) * t->nflags), "cudaMemset flags");
  CK(cudaMalloc(&t->d_status, sizeof(LaunchStatus)), "cudaMalloc status");
  CK(cudaMemset(t->d_status, 0, sizeof(LaunchStatus)), "cudaMemset status");
  CK(cudaMallocHost(&t->h_status, sizeof(LaunchStatus)), "cudaMallocHost status");
  CK(cudaMalloc(&t->d_map, sizeof(int) * 5), "cudaMalloc cluster map");
  std::memset(t->h_status, 0, sizeof(LaunchStatus));
  t->nblocks = std::max({1, residual_blocks(h.N), rowgrid_blocks(h.N)});
  {
    std::vector<int> chunks(residual_chunks(h.N));
    residual_chunk_list(h.N, chunks.data());
    CK(cudaMalloc(&t->d_chunks, sizeof(int) * std::max<size_t>(chunks.size(), 1)), "cudaMalloc residual chunks");
    if (!chunks.empty())
      CK(cudaMemcpy(t->d_chunks, chunks.data(), sizeof(int) * chunks.size(), cudaMemcpyHostToDevice),
         "upload residual chunks");
    t->dev.chunks = t->d_chunks;
    t->dev.nchunks = (int)chunks.size();
    std::vector<int> strips(residual_strips(h.N));
    residual_strip_list(h.N, strips.data());
    CK(cudaMalloc(&t->d_strips, sizeof(int) * std::max<size_t>(strips.size(), 1)), "cudaMalloc residual strips");
    if (!strips.empty())
      CK(cudaMemcpy(t->d_strips, strips.data(), sizeof(int) * strips.size(), cudaMemcpyHostToDevice),
         "upload residual strips");
    t->dev.strips = t->d_strips;
    t->dev.nstrips = (int)strips.size();
  }
  CK(cudaMalloc(&t->d_dev, sizeof(DevTet)), "cudaMalloc tet");
  // band kernels: measured faster than the slab kernels from level 9 on
  // (L7/L8/L9 MIXED sweeps: 0.78/1.77/10.2 ms slab, 1.10/2.19/6.0 ms band)
  t->use_band = t->precision != ILU_F64 && wave_uses_registers(t->kind(), h.dx) &&
                (t->kernel_choice == ILU_KERNEL_BAND || (t->kernel_choice == ILU_KERNEL_AUTO && h.L >= 9));
  if (t->use_band) {
    ilu_status bs = upload_band(t, t->requested_slabs);
    if (bs != ILU_OK) return bs;
  }
  // packed kernels: one CTA (level 8: a cluster of two) per tet (see
  // packed.h); measured faster than the slab kernels for a single tet up to
  // level 6 (F32 sweeps at L5/L6/L7/L8: 0.086/0.21/0.70/4.87 ms packed,
  // 0.14/0.30/0.63/1.73 ms slab), and the batch kernel of choice (no waits
  // between tets)
  t->use_packed = !t->use_band && t->precision != ILU_F64 && h.dx <= kPackedMaxDegree &&
                  h.L <= kPackedMaxLevel &&
                  (t->kernel_choice == ILU_KERNEL_PACKED || (t->kernel_choice == ILU_KERNEL_AUTO && h.L <= 6));
  if (t->use_packed) {
    ilu_status ps = upload_packed(t);
    if (ps != ILU_OK) return ps;
  }
  CK(cudaMalloc(&t->d_partials, sizeof(double) * t->nblocks), "cudaMalloc partials");
  t->norms_cap = 0;
  DevTet &d = t->dev;
  d.L = h.L; d.N = h.N; d.h = h.h; d.dx = h.dx; d.rstride = h.rstride;
  d.const_kappa = h.const_kappa ? 1 : 0;
  d.tabF = t->d_tabF; d.tabB = t->d_tabB; d.kappa = t->d_kappa; d.w = t->d_w; d.flags = t->d_flags;
  std::memcpy(d.A15, h.A15, sizeof(d.A15));
  std::memcpy(d.Wstar, h.Wstar, sizeof(d.Wstar));
  d.astore = nullptr;
  d.astride = (int64_t)nn;
  d.bnd = nullptr;
  d.bnd_off = nullptr;
  if (h.boundary == ILU_BOUNDARY_V1) {
    const size_t nrec = h.bndL.size() / 8;
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    CK(cudaMalloc(&t->d_bnd, std::max<size_t>(nrec, 1) * 8 * es), "cudaMalloc boundary factors");
    CK(cudaMalloc(&t->d_bnd_off, h.bnd_rowoff.size() * sizeof(int)), "cudaMalloc boundary offsets");
    if (f64) {
      if (nrec) CK(cudaMemcpy(t->d_bnd, h.bndL.data(), nrec * 8 * es, cudaMemcpyHostToDevice), "upload boundary factors");
    } else {
      std::vector<float> f(h.bndL.begin(), h.bndL.end());
      if (nrec) CK(cudaMemcpy(t->d_bnd, f.data(), nrec * 8 * es, cudaMemcpyHostToDevice), "upload boundary factors");
    }
    CK(cudaMemcpy(t->d_bnd_off, h.bnd_rowoff.data(), h.bnd_rowoff.size() * sizeof(int), cudaMemcpyHostToDevice),
       "upload boundary offsets");
    d.bnd = t->d_bnd;
    d.bnd_off = t->d_bnd_off;
  }
  if (!h.const_kappa) {
    const bool a32 = t->precision == ILU_F32;
    const size_t abytes = (size_t)(kNumDirs - 1) * nn * (a32 ? sizeof(float) : sizeof(double));
    const bool store = t->stencil_choice == ILU_STENCIL_STORED ||
                       (t->stencil_choice == ILU_STENCIL_AUTO && abytes <= ((size_t)4 << 30));
    if (store) {
      CK(cudaMalloc(&t->d_astore, abytes), "cudaMalloc stored stencils");
      CK(launch_stencil_store(d, t->d_astore, a32, cudaStreamPerThread), "stencil assembly launch");
      CK(cudaStreamSynchronize(cudaStreamPerThread), "stencil assembly");
      d.astore = t->d_astore;
    }
  }
  d.valsF = d.valsB = nullptr;
  if (t->tabulate) {
    const size_t vbytes = nn * 8 * sizeof(double);
    CK(cudaMalloc(&t->d_valsF, vbytes), "cudaMalloc tabulated values");
    CK(cudaMalloc(&t->d_valsB, vbytes), "cudaMalloc tabulated values");
    CK(cudaMemset(t->d_valsF, 0, vbytes), "cudaMemset tabulated values");
    CK(cudaMemset(t->d_valsB, 0, vbytes), "cudaMemset tabulated values");
    CK(launch_tabulate(d, t->d_valsF, t->d_valsB, cudaStreamPerThread), "tabulation launch");
    CK(cudaStreamSynchronize(cudaStreamPerThread), "tabulation");
    d.valsF = t->d_valsF;
    d.valsB = t->d_valsB;
  }
  return choose_clusters(t);
}

ilu_status upload_tables(ilu_tet t) {
  HostTet &h = t->host;
  CK(cudaSetDevice(t->device), "cudaSetDevice");
  const bool f64 = t->precision == ILU_F64;
  const size_t es = f64 ? sizeof(double) : sizeof(float);
  const size_t nf = f64 ? h.tabF64.size() : h.tabF32.size(), nb = f64 ? h.tabB64.size() : h.tabB32.size();
  if (nf)
    CK(cudaMemcpy(t->d_tabF, f64 ? (const void *)h.tabF64.data() : (const void *)h.tabF32.data(), nf * es,
                  cudaMemcpyHostToDevice), "upload tables");
  if (nb)
    CK(cudaMemcpy(t->d_tabB, f64 ? (const void *)h.tabB64.data() : (const void *)h.tabB32.data(), nb * es,
                  cudaMemcpyHostToDevice), "upload tables");
  if (t->use_packed) {  // so do the packed kernels' compact copies
    ilu_status ps = upload_packed_tables(t);
    if (ps != ILU_OK) return ps;
  }
  if (t->tabulate) {  // the tabulated values follow the new polynomials
    CK(launch_tabulate(t->dev, t->d_valsF, t->d_valsB, cudaStreamPerThread), "tabulation launch");
    CK(cudaStreamSynchronize(cudaStreamPerThread), "tabulation");
  }
  return ILU_OK;
}

// the surrogate pivot inverse must be positive everywhere for L~ D~ L~^T to
// be symmetric positive definite (every interior point checked, face layers
// shared out over host threads)
ilu_status check_surrogate(const HostTet &h) {
  const int N = h.N;
  const int nth = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
  std::vector<char> bad(nth, 0);
  auto work = [&](int k) {
    for (int z = 1 + k; z <= N - 3 && !bad[k]; z += nth)
      for (int y = 1; y <= N - 2 - z; ++y)
        for (int x = 1; x <= N - 1 - y - z; ++x) {
          double v[8];
          host_eval_tables(h, x, y, z, v);
          if (!(v[7] > 0.0) || !std::isfinite(v[7])) {
            bad[k] = 1;
            return;
          }
        }
  };
  std::vector<std::thread> pool;
  for (int k = 0; k < nth; ++k) pool.emplace_back(work, k);
  for (auto &th : pool) th.join();
  for (char b : bad)
    if (b) return fail(ILU_ESINGULAR, "surrogate 1/D is not positive at an interior point");
  return ILU_OK;
}

ilu_status ensure_norms(ilu_tet t, int n) {
  if (t->norms_cap >= n) return ILU_OK;
  cudaFree(t->d_norms);
  t->d_norms = nullptr;
  int cap = std::max(n, 64);
  CK(cudaMalloc(&t->d_norms, sizeof(double) * cap), "cudaMalloc norms");
  t->norms_cap = cap;
  return ILU_OK;
}

ilu_status check_usable(ilu_tet t) {
  if (!t) return fail(ILU_EINVAL, "null handle");
  if (t->device < 0) return fail(ILU_ENODEV, "host-only handle has no device part");
  if (t->failed) return fail(ILU_ECUDA, "handle failed earlier; destroy it");
  return ILU_OK;
}

ilu_status read_status(ilu_tet t, cudaStream_t st) {
  CK(cudaMemcpyAsync(t->h_status, t->d_status, sizeof(LaunchStatus), cudaMemcpyDeviceToHost, st), "status copy");
  CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  if (t->h_status->code != 0) {
    t->failed = true;
    return fail(ILU_ETIMEOUT, "a bounded device wait ran out (slab " + std::to_string(t->h_status->where) +
                                  ", level " + std::to_string(t->h_status->level) + ")");
  }
  return ILU_OK;
}

cudaEvent_t pool_event(ilu_tet t) {
  if (!t->ev_pool.empty()) {
    cudaEvent_t e = t->ev_pool.back();
    t->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// bracket one launch with events when tracing is on
struct Traced {
  ilu_tet t;
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  Traced(ilu_tet t_, int k, cudaStream_t s) : t(t_), kind(k), st(s) {
    t->launches++;
    if (t->prof) {
      a = pool_event(t);
      cudaEventRecord(a, st);
    }
  }
  ~Traced() {
    if (a) {
      cudaEvent_t b = pool_event(t);
      cudaEventRecord(b, st);
      t->ev_used.push_back({kind, a, b});
    }
  }
};

// one sweep on device vectors: residual into w, forward, backward with x += w
ilu_status sweep(ilu_tet t, void *x, const void *b, double *d_norm_out, cudaStream_t st) {
  CK(cudaMemsetAsync(t->d_flags, 0, sizeof(int) * t->nflags, st), "reset flags");
  if (t->use_band) {
    {
      Traced tr(t, 0, st);
      CK(launch_band_in(t->kind(), 0, t->d_dev, t->band_tprefix, 1, t->band_ntiles, nullptr, nullptr, x, b,
                        t->d_partials, st),
         "residual launch");
    }
    if (d_norm_out) {
      t->launches++;
      CK(launch_norm_finish(t->d_partials, t->band_ntiles, d_norm_out, st), "norm launch");
    }
    {
      Traced tr(t, 1, st);
      CK(launch_band_sub(true, t->bl, t->d_status, t->max_spins, st), "forward launch");
    }
    {
      Traced tr(t, 2, st);
      CK(launch_band_sub(false, t->bl, t->d_status, t->max_spins, st), "backward launch");
      t->launches++;
      CK(launch_band_update(t->kind(), t->d_dev, t->band_tprefix, 1, t->band_ntiles, nullptr, x, st), "update launch");
    }
    return ILU_OK;
  }
  int used = 0;
  {
    Traced tr(t, 0, st);
    CK(launch_residual(t->dev, t->kind(), x, b, t->d_w, t->d_partials, t->nblocks, &used, st, t->use_packed),
       "residual launch");
  }
  if (d_norm_out) {
    t->launches++;
    CK(launch_norm_finish(t->d_partials, used, d_norm_out, st), "norm launch");
  }
  if (t->use_packed) {  // forward and backward substitution in one launch (traced as the forward)
    {
      Traced tr(t, 1, st);
      CK(launch_packed(t->pl, st), "packed substitution launch");
    }
    Traced tr(t, 2, st);  // x += w (traced as the backward)
    CK(launch_packed_io(0, t->precision != ILU_F32, t->d_dev, nullptr, residual_blocks(t->host.N), nullptr, x, st),
       "update launch");
    return ILU_OK;
  }
  {
    Traced tr(t, 1, st);
    CK(launch_forward(t->wl, t->d_status, t->max_spins, st), "forward launch");
  }
  {
    Traced tr(t, 2, st);
    WaveLaunch L = t->wl;
    L.map_b.x0 = x;
    CK(launch_backward(L, t->d_status, t->max_spins, st), "backward launch");
  }
  return ILU_OK;
}

// apply the preconditioner: z = C~^{-1} r on the interior (z's boundary 0)
ilu_status precond(ilu_tet t, const void *r, void *z, cudaStream_t st) {
  const long long n = (long long)t->nnodes();
  const bool vf64 = t->precision != ILU_F32;   // Krylov vectors
  const bool wf64 = t->precision == ILU_F64;   // sweep scratch
  CK(cudaMemsetAsync(t->d_flags, 0, sizeof(int) * t->nflags, st), "reset flags");
  if (t->use_band) {
    t->launches++;
    CK(launch_band_in(t->kind(), 1, t->d_dev, t->band_tprefix, 1, t->band_ntiles, nullptr, nullptr, r, nullptr,
                      nullptr, st),
       "copy launch");
    CK(cudaMemsetAsync(z, 0, n * t->elem(), st), "clear z");
    {
      Traced tr(t, 1, st);
      CK(launch_band_sub(true, t->bl, t->d_status, t->max_spins, st), "forward launch");
    }
    {
      Traced tr(t, 2, st);
      CK(launch_band_sub(false, t->bl, t->d_status, t->max_spins, st), "backward launch");
      t->launches++;
      CK(launch_band_update(t->kind(), t->d_dev, t->band_tprefix, 1, t->band_ntiles, nullptr, z, st), "update launch");
    }
    return ILU_OK;
  }
  if (t->use_packed) {  // r into the packed array, the substitutions, z = their result
    const int nb = residual_blocks(t->host.N);
    t->launches++;
    CK(launch_packed_io(1, vf64, t->d_dev, nullptr, nb, nullptr, const_cast<void *>(r), st), "copy launch");
    CK(cudaMemsetAsync(z, 0, n * t->elem(), st), "clear z");
    {
      Traced tr(t, 1, st);
      CK(launch_packed(t->pl, st), "packed substitution launch");
    }
    Traced tr(t, 2, st);
    CK(launch_packed_io(0, vf64, t->d_dev, nullptr, nb, nullptr, z, st), "update launch");
    return ILU_OK;
  }
  CK(launch_copy(vf64, wf64, r, t->d_w, n, st), "copy launch");
  CK(cudaMemsetAsync(z, 0, n * t->elem(), st), "clear z");
  {
    Traced tr(t, 1, st);
    CK(launch_forward(t->wl, t->d_status, t->max_spins, st), "forward launch");
  }
  {
    Traced tr(t, 2, st);
    WaveLaunch L = t->wl;
    L.map_b.x0 = z;
    CK(launch_backward(L, t->d_status, t->max_spins, st), "backward launch");
  }
  return ILU_OK;
}

ilu_status ensure_krylov(ilu_tet t) {
  if (t->d_r) return ILU_OK;
  const size_t bytes = t->nnodes() * t->elem();
  for (void **v : {&t->d_r, &t->d_z, &t->d_p, &t->d_q, &t->d_zero}) {
    CK(cudaMalloc(v, bytes), "cudaMalloc Krylov vectors");
    CK(cudaMemset(*v, 0, bytes), "cudaMemset Krylov vectors");
  }
  CK(cudaMalloc(&t->d_dot, sizeof(double) * kDotPartials), "cudaMalloc dot partials");
  CK(cudaMalloc(&t->d_scal, sizeof(double) * 8), "cudaMalloc scalars");
  CK(cudaMallocHost(&t->h_scal, sizeof(double) * 8), "cudaMallocHost scalars");
  return ILU_OK;
}

// read n device scalars (synchronising the stream)
ilu_status read_scalars(ilu_tet t, int n, cudaStream_t st) {
  CK(cudaMemcpyAsync(t->h_scal, t->d_scal, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "scalar copy");
  CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  if (t->h_status && t->h_status->code) return fail(ILU_ETIMEOUT, "a bounded device wait ran out");
  return ILU_OK;
}

}  // namespace

namespace ilu {
// read-only view of a handle's device data for ilu_residual_noalloc
const DevTet *tet_dev_view(ilu_tet t, int *device, int *precision, size_t *nnodes) {
  if (!t) return nullptr;
  *device = t->device;
  *precision = t->precision;
  *nnodes = t->nnodes();
  return t->device >= 0 ? &t->dev : nullptr;
}
ilu_status tet_acquire(ilu_tet t, std::unique_lock<std::mutex> *lk) {
  const ilu_status st = check_usable(t);
  if (st != ILU_OK) return st;
  *lk = std::unique_lock<std::mutex>(t->mu);
  return t->failed ? fail(ILU_ECUDA, "handle failed earlier; destroy it") : ILU_OK;
}
void tet_mark_failed(ilu_tet t) { t->failed = true; }
void set_last_error(const std::string &msg) { g_err = msg; }
bool tet_view(ilu_tet t, TetView *v) {
  if (!t || t->device < 0) return false;
  v->dev = &t->dev;
  v->N = t->host.N;
  v->dx = t->host.dx;
  v->rstride = t->host.rstride;
  v->device = t->device;
  v->precision = t->precision;
  v->kind = t->kind();
  v->reg = t->wave_reg();
  v->nnodes = t->nnodes();
  v->failed = t->failed;
  v->packed = t->use_packed;
  v->packed_steps = t->use_packed ? 2 * t->dev.pk.nsteps : 0;
  v->packed_q = t->use_packed ? t->pl.q : 0;
  v->packed_cl = t->use_packed ? t->pl.cl : 0;
  return true;
}
WaveGeom wave_geom(int N, int kind, int dxp, int reg, bool fwd, int requested) {
  return pick_geom(N, kind, dxp, reg, fwd, requested);
}
ilu_status tet_sweeps(ilu_tet t, void *x, const void *b, int n, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(t->mu);
  for (int k = 0; k < n; ++k) {
    ilu_status st = sweep(t, x, b, nullptr, s);
    if (st != ILU_OK) {
      t->failed = true;
      return st;
    }
  }
  return ILU_OK;
}
ilu_status tet_residual(ilu_tet t, const void *x, const void *b, void *r, double *d_norm, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(t->mu);
  const int vkind = t->precision == ILU_F32 ? kSweepF32 : kSweepF64;
  int used = 0;
  CK(launch_residual(t->dev, vkind, x, b, r, t->d_partials, t->nblocks, &used, s), "residual launch");
  if (d_norm) CK(launch_norm_finish(t->d_partials, used, d_norm, s), "norm launch");
  return ILU_OK;
}
ilu_status tet_check(ilu_tet t, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(t->mu);
  return read_status(t, s);
}
}  // namespace ilu

extern "C" {

ilu_status ilu_opts_default(ilu_opts *o) {
  if (!o) return fail(ILU_EINVAL, "null opts");
  o->deg[0] = o->deg[1] = o->deg[2] = -1;
  o->sample_level = -1;
  o->ridge = -1.0;
  o->precision = ILU_MIXED;
  o->slabs = 0;
  o->device = 0;
  o->max_wait_spins = 0;
  o->kernel = ILU_KERNEL_AUTO;
  o->factor = ILU_FACTOR_ILU0;
  o->stencil = ILU_STENCIL_AUTO;
  o->orient = ILU_ORIENT_GIVEN;
  o->boundary = ILU_BOUNDARY_V2;
  o->max_cluster = 0;
  o->values = ILU_VALUES_AUTO;
  return ILU_OK;
}

const char *ilu_last_error(void) { return g_err.c_str(); }
const char *ilu_version(void) { return "gb300-surrogate-ilu 0.1 (sm_103a)"; }

size_t ilu_num_nodes(int level) {
  if (level < 2 || level > 10) return 0;
  return (size_t)grid_nodes(1 << level);
}

size_t ilu_num_interior(int level) {
  if (level < 2 || level > 10) return 0;
  return (size_t)grid_interior(1 << level);
}

long long ilu_index(int level, int x, int y, int z) {
  if (level < 2 || level > 10) return -1;
  const int N = 1 << level;
  if (!in_grid(N, x, y, z)) return -1;
  return (long long)grid_index(N, x, y, z);
}

ilu_status ilu_setup(const double macro_tet[12], int level, const ilu_coeff *coeff, int poly_degree,
                     const ilu_opts *opts, ilu_tet *out) {
  ilu::DeviceRestore keep_device;
  if (!out) return fail(ILU_EINVAL, "null output handle");
  *out = nullptr;
  if (!macro_tet) return fail(ILU_EINVAL, "null macro_tet");
  ilu_opts o;
  ilu_opts_default(&o);
  if (opts) o = *opts;
  if (o.precision < 0 || o.precision > 2) return fail(ILU_EINVAL, "unknown precision");
  if (o.kernel < ILU_KERNEL_AUTO || o.kernel > ILU_KERNEL_PACKED) return fail(ILU_EINVAL, "unknown kernel choice");
  if (o.kernel == ILU_KERNEL_PACKED && (level > kPackedMaxLevel || o.precision == ILU_F64))
    return fail(ILU_EINVAL, "the packed kernels take FP32/MIXED sweeps up to level 8");
  if (o.kernel == ILU_KERNEL_PACKED && (o.deg[0] >= 0 ? o.deg[0] : poly_degree) > kPackedMaxDegree)
    return fail(ILU_EINVAL, "the packed kernels take row (x) degrees up to 6");
  if (o.factor != ILU_FACTOR_ILU0 && o.factor != ILU_FACTOR_SGS) return fail(ILU_EINVAL, "unknown factor choice");
  if (o.stencil < ILU_STENCIL_AUTO || o.stencil > ILU_STENCIL_STORED) return fail(ILU_EINVAL, "unknown stencil choice");
  if (o.orient != ILU_ORIENT_GIVEN && o.orient != ILU_ORIENT_LFA) return fail(ILU_EINVAL, "unknown orientation choice");
  if (o.boundary != ILU_BOUNDARY_V2 && o.boundary != ILU_BOUNDARY_V1) return fail(ILU_EINVAL, "unknown boundary variant");
  if (o.values < ILU_VALUES_AUTO || o.values > ILU_VALUES_TABULATED) return fail(ILU_EINVAL, "unknown values choice");
  if (o.values == ILU_VALUES_TABULATED && o.precision != ILU_F64)
    return fail(ILU_EINVAL, "tabulated surrogate values are an FP64 option");
  if (o.values == ILU_VALUES_TABULATED && level > kTabulatedMaxLevel)
    return fail(ILU_EINVAL, "tabulated surrogate values need level <= 9");
  int perm[4] = {0, 1, 2, 3};
  if (o.orient == ILU_ORIENT_LFA) {
    ilu_status ls = ilu_lfa_order(macro_tet, perm, nullptr, nullptr);
    if (ls != ILU_OK) return ls;
  }
  double Pv[12];
  for (int i = 0; i < 4; ++i)
    for (int c = 0; c < 3; ++c) Pv[3 * i + c] = macro_tet[3 * perm[i] + c];
  int deg[3];
  for (int c = 0; c < 3; ++c) deg[c] = o.deg[c] >= 0 ? o.deg[c] : poly_degree;
  ilu_tet t = new (std::nothrow) ilu_tet_s;
  if (!t) return fail(ILU_ENOMEM, "out of host memory");
  t->precision = o.precision;
  t->device = o.device;
  std::memcpy(t->perm, perm, sizeof(perm));
  t->max_spins = o.max_wait_spins > 0 ? o.max_wait_spins : kDefaultSpins;
  std::string err;
  ilu_status st;
  try {
    t->host.factor = o.factor;
    t->host.boundary = o.boundary;
    st = host_setup(t->host, Pv, level, coeff, deg, o.sample_level, o.ridge, err);
  } catch (const std::bad_alloc &) {
    st = ILU_ENOMEM;
    err = "out of host memory during set-up";
  }
  if (st != ILU_OK) {
    delete t;
    return fail(st, err);
  }
  st = check_surrogate(t->host);
  if (st != ILU_OK) {
    delete t;
    return st;
  }
  if (t->device >= 0) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= t->device) {
      cudaGetLastError();
      delete t;
      return fail(ILU_ENODEV, "no CUDA device with that ordinal");
    }
    {
      const size_t vbytes = 2 * (size_t)grid_nodes(1 << level) * 8 * sizeof(double);
      t->tabulate = o.precision == ILU_F64 && level <= kTabulatedMaxLevel &&
                    (o.values == ILU_VALUES_TABULATED || (o.values == ILU_VALUES_AUTO && vbytes <= ((size_t)4 << 30)));
    }
    choose_geometry(t, o.slabs);
    t->requested_slabs = o.slabs;
    t->kernel_choice = o.kernel;
    t->stencil_choice = o.stencil;
    t->max_cluster = o.max_cluster;
    st = upload(t);
    if (st != ILU_OK) {
      free_device(t);
      delete t;
      return st;
    }
  }
  *out = t;
  return ILU_OK;
}

ilu_status ilu_destroy(ilu_tet t) {
  ilu::DeviceRestore keep_device;
  if (!t) return ILU_OK;
  free_device(t);
  delete t;
  return ILU_OK;
}

ilu_status ilu_vertex_order(ilu_tet t, int perm[4]) {
  if (!t || !perm) return fail(ILU_EINVAL, "null argument");
  std::memcpy(perm, t->perm, sizeof(t->perm));
  return ILU_OK;
}

size_t ilu_surrogate_size(ilu_tet t) { return t ? t->host.coefs.size() : 0; }

ilu_status ilu_export_surrogate(ilu_tet t, double *coefs, size_t n) {
  if (!t || !coefs) return fail(ILU_EINVAL, "null argument");
  if (n < t->host.coefs.size()) return fail(ILU_EINVAL, "output too small");
  std::memcpy(coefs, t->host.coefs.data(), sizeof(double) * t->host.coefs.size());
  return ILU_OK;
}

ilu_status ilu_import_surrogate(ilu_tet t, const double *coefs, size_t n) {
  ilu::DeviceRestore keep_device;
  if (!t || !coefs) return fail(ILU_EINVAL, "null argument");
  if (n != t->host.coefs.size()) return fail(ILU_EINVAL, "coefficient count does not match the handle's degrees");
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(coefs[i])) return fail(ILU_EINVAL, "non-finite coefficient");
  std::lock_guard<std::mutex> lk(t->mu);
  if (t->device >= 0 && t->failed) return fail(ILU_ECUDA, "handle failed earlier; destroy it");
  std::vector<double> old = t->host.coefs;
  std::memcpy(t->host.coefs.data(), coefs, sizeof(double) * n);
  build_row_tables(t->host);
  ilu_status st = check_surrogate(t->host);
  if (st != ILU_OK) {
    t->host.coefs = old;
    build_row_tables(t->host);
    return st;
  }
  if (t->device >= 0) {
    st = upload_tables(t);  // device tables (and tabulated values) now disagree with the host: unusable
    if (st != ILU_OK) t->failed = true;
    return st;
  }
  return ILU_OK;
}

ilu_status ilu_eval_surrogate(ilu_tet t, int x, int y, int z, double out[8]) {
  if (!t || !out) return fail(ILU_EINVAL, "null argument");
  if (!in_interior(t->host.N, x, y, z)) return fail(ILU_EINVAL, "point is not interior");
  host_eval_tables(t->host, x, y, z, out);
  return ILU_OK;
}

ilu_status ilu_exact_factor(ilu_tet t, int x, int y, int z, double out[8]) {
  if (!t || !out) return fail(ILU_EINVAL, "null argument");
  const HostTet &h = t->host;
  if (!h.keep_exact) return fail(ILU_EINVAL, "exact factors are kept only for level <= 7");
  if (!in_interior(h.N, x, y, z)) return fail(ILU_EINVAL, "point is not interior");
  // interior lexicographic number of (x,y,z)
  const int N = h.N;
  int64_t i = 0;
  for (int zz = 1; zz < z; ++zz)
    for (int yy = 1; yy <= N - 2 - zz; ++yy) i += N - 1 - yy - zz;
  for (int yy = 1; yy < y; ++yy) i += N - 1 - yy - z;
  i += x - 1;
  const int64_t nint = grid_interior(N);
  for (int d = 0; d < 7; ++d) out[d] = h.exactL[(size_t)d * nint + i];
  out[7] = h.exactD[i];
  return ILU_OK;
}

ilu_status ilu_stencil(ilu_tet t, int x, int y, int z, double out[15]) {
  if (!t || !out) return fail(ILU_EINVAL, "null argument");
  if (!in_interior(t->host.N, x, y, z)) return fail(ILU_EINVAL, "point is not interior");
  host_stencil(t->host, x, y, z, out);
  return ILU_OK;
}

ilu_status ilu_smooth(ilu_tet t, void *x, const void *b, int sweeps, void *stream, double *res_norms) {
  ilu::DeviceRestore keep_device;
  ilu_status st = check_usable(t);
  if (st != ILU_OK) return st;
  if (!x || !b) return fail(ILU_EINVAL, "null vector");
  if (sweeps < 0) return fail(ILU_EINVAL, "negative sweep count");
  if (sweeps == 0) return ILU_OK;
  std::lock_guard<std::mutex> lk(t->mu);
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(t->device), "cudaSetDevice");
  if (res_norms) {
    st = ensure_norms(t, sweeps);
    if (st != ILU_OK) return st;
  }
  for (int k = 0; k < sweeps; ++k) {
    st = sweep(t, x, b, res_norms ? t->d_norms + k : nullptr, s);
    if (st != ILU_OK) { t->failed = true; return st; }
  }
  if (res_norms) {
    CK(cudaMemcpyAsync(res_norms, t->d_norms, sizeof(double) * sweeps, cudaMemcpyDeviceToHost, s), "norms copy");
    return read_status(t, s);
  }
  return ILU_OK;
}

ilu_status ilu_smooth_host(ilu_tet t, void *x_host, const void *b_host, int sweeps, double *res_norms) {
  ilu::DeviceRestore keep_device;
  ilu_status st = check_usable(t);
  if (st != ILU_OK) return st;
  if (!x_host || !b_host) return fail(ILU_EINVAL, "null vector");
  const size_t bytes = t->nnodes() * t->elem();
  {
    std::lock_guard<std::mutex> lk(t->mu);
    CK(cudaSetDevice(t->device), "cudaSetDevice");
    if (!t->d_xs) CK(cudaMalloc(&t->d_xs, bytes), "cudaMalloc staging");
    if (!t->d_bs) CK(cudaMalloc(&t->d_bs, bytes), "cudaMalloc staging");
    CK(cudaMemcpy(t->d_xs, x_host, bytes, cudaMemcpyHostToDevice), "copy x");
    CK(cudaMemcpy(t->d_bs, b_host, bytes, cudaMemcpyHostToDevice), "copy b");
  }
  st = ilu_smooth(t, t->d_xs, t->d_bs, sweeps, nullptr, res_norms);
  if (st != ILU_OK) return st;
  std::lock_guard<std::mutex> lk(t->mu);
  CK(cudaMemcpy(x_host, t->d_xs, bytes, cudaMemcpyDeviceToHost), "copy x back");
  if (!res_norms) return read_status(t, nullptr);
  return ILU_OK;
}

ilu_status ilu_residual(ilu_tet t, const void *x, const void *b, void *r, double *norm2, void *stream) {
  ilu::DeviceRestore keep_device;
  ilu_status st = check_usable(t);
  if (st != ILU_OK) return st;
  if (!x || !b) return fail(ILU_EINVAL, "null vector");
  std::lock_guard<std::mutex> lk(t->mu);
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(t->device), "cudaSetDevice");
  // the residual kernel writes interior entries only: clear r's boundary
  void *dst = r ? r : t->d_w;
  const int kind = t->precision == ILU_F32 ? kSweepF32 : kSweepF64;
  if (r) CK(cudaMemsetAsync(r, 0, t->nnodes() * t->elem(), s), "clear r");
  int used = 0;
  if (!r && t->precision == ILU_MIXED) {
    // scratch holds floats in MIXED mode: compute the norm through the mixed kernel
    CK(launch_residual(t->dev, kSweepMixed, x, b, t->d_w, t->d_partials, t->nblocks, &used, s), "residual launch");
  } else {
    CK(launch_residual(t->dev, kind, x, b, dst, t->d_partials, t->nblocks, &used, s), "residual launch");
  }
  if (norm2) {
    st = ensure_norms(t, 1);
    if (st != ILU_OK) return st;
    CK(launch_norm_finish(t->d_partials, used, t->d_norms, s), "norm launch");
    CK(cudaMemcpyAsync(norm2, t->d_norms, sizeof(double), cudaMemcpyDeviceToHost, s), "norm copy");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  }
  return ILU_OK;
}

ilu_status ilu_solve(ilu_tet t, void *x, const void *b, int method, double rtol, int max_iter, void *stream,
                     int *iters, double *rel_res) {
  ilu::DeviceRestore keep_device;
  ilu_status st = check_usable(t);
  if (st != ILU_OK) return st;
  if (!x || !b) return fail(ILU_EINVAL, "null vector");
  if (method == ILU_MG_VCYCLE || method == ILU_MG_PCG) return fail(ILU_EINVAL, "multigrid methods need ilu_mg_solve");
  if (method != ILU_RICHARDSON && method != ILU_PCG) return fail(ILU_EINVAL, "unknown method");
  if (!(rtol >= 0.0) || max_iter < 0) return fail(ILU_EINVAL, "bad tolerance or iteration limit");
  std::lock_guard<std::mutex> lk(t->mu);
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaSetDevice(t->device), "cudaSetDevice");
  st = ensure_krylov(t);
  if (st != ILU_OK) return st;
  const int N = t->host.N;
  const long long n = (long long)t->nnodes();
  const bool vf64 = t->precision != ILU_F32;
  const int vkind = vf64 ? kSweepF64 : kSweepF32;  // residual into a Krylov-typed vector
  if (iters) *iters = 0;
  if (rel_res) *rel_res = 0.0;
  // ||b|| over the interior
  CK(cudaMemcpyAsync(t->h_status, t->d_status, sizeof(LaunchStatus), cudaMemcpyDeviceToHost, s), "status copy");
  CK(launch_interior_norm(N, vf64, b, t->d_partials, t->nblocks, t->d_scal, s), "norm launch");
  st = read_scalars(t, 1, s);
  if (st != ILU_OK) return st;
  double bn = t->h_scal[0];
  if (bn == 0.0) bn = 1.0;
  auto residual_norm = [&](double &rel) -> ilu_status {  // r = b - A x, rel = ||r|| / ||b||
    int used = 0;
    CK(launch_residual(t->dev, vkind, x, b, t->d_r, t->d_partials, t->nblocks, &used, s), "residual launch");
    CK(launch_norm_finish(t->d_partials, used, t->d_scal, s), "norm launch");
    CK(cudaMemcpyAsync(t->h_status, t->d_status, sizeof(LaunchStatus), cudaMemcpyDeviceToHost, s), "status copy");
    ilu_status e = read_scalars(t, 1, s);
    rel = t->h_scal[0] / bn;
    return e;
  };
  double rel = 0.0;
  if (method == ILU_RICHARDSON) {
    // defect correction: r in FP64 (MIXED/F64), correction C~^{-1} r in the sweep precision
    for (int it = 0;; ++it) {
      st = residual_norm(rel);
      if (st != ILU_OK) { t->failed = true; return st; }
      if (iters) *iters = it;
      if (rel_res) *rel_res = rel;
      if (rel <= rtol) return ILU_OK;
      if (it == max_iter) return fail(ILU_ENOTCONV, "Richardson iteration reached max_iter");
      st = precond(t, t->d_r, t->d_z, s);
      if (st != ILU_OK) { t->failed = true; return st; }
      CK(launch_axpy(vf64, x, t->d_z, 1.0, n, s), "axpy launch");
    }
  }
  // preconditioned conjugate gradients on the interior system
  st = residual_norm(rel);
  if (st != ILU_OK) { t->failed = true; return st; }
  double rz_old = 0.0;
  for (int it = 0;; ++it) {
    if (iters) *iters = it;
    if (rel_res) *rel_res = rel;
    if (rel <= rtol) return ILU_OK;
    if (it == max_iter) return fail(ILU_ENOTCONV, "PCG reached max_iter");
    st = precond(t, t->d_r, t->d_z, s);
    if (st != ILU_OK) { t->failed = true; return st; }
    CK(launch_dot(vf64, t->d_r, t->d_z, n, t->d_dot, t->d_scal, s), "dot launch");
    st = read_scalars(t, 1, s);
    if (st != ILU_OK) { t->failed = true; return st; }
    const double rz = t->h_scal[0];
    if (it == 0)
      CK(launch_copy(vf64, vf64, t->d_z, t->d_p, n, s), "copy launch");
    else
      CK(launch_xpay(vf64, t->d_p, t->d_z, rz / rz_old, n, s), "xpay launch");
    rz_old = rz;
    // q = -A p (the residual kernel with b = 0; p vanishes on the boundary)
    int used = 0;
    CK(launch_residual(t->dev, vkind, t->d_p, t->d_zero, t->d_q, t->d_partials, t->nblocks, &used, s),
       "matvec launch");
    CK(launch_dot(vf64, t->d_p, t->d_q, n, t->d_dot, t->d_scal, s), "dot launch");
    st = read_scalars(t, 1, s);
    if (st != ILU_OK) { t->failed = true; return st; }
    const double pAp = -t->h_scal[0];
    if (!(pAp > 0.0)) return fail(ILU_ESINGULAR, "PCG met a non-positive curvature");
    const double alpha = rz / pAp;
    CK(launch_axpy(vf64, x, t->d_p, alpha, n, s), "axpy launch");
    CK(launch_axpy(vf64, t->d_r, t->d_q, alpha, n, s), "axpy launch");  // r -= alpha A p
    CK(launch_dot(vf64, t->d_r, t->d_r, n, t->d_dot, t->d_scal, s), "dot launch");
    st = read_scalars(t, 1, s);
    if (st != ILU_OK) { t->failed = true; return st; }
    rel = std::sqrt(std::max(t->h_scal[0], 0.0)) / bn;
  }
}

ilu_status ilu_packed_schedule(int level, int forward, int lanes, int quantum, int *nsteps, int *lanes_out,
                               int *entries, int *lane_off) {
  if (!nsteps || !lanes_out) return fail(ILU_EINVAL, "null argument");
  if (level < 2 || level > kPackedMaxLevel) return fail(ILU_EINVAL, "the packed schedules cover levels 2 to 8");
  if (lanes < 0 || lanes > 1016) return fail(ILU_EINVAL, "lanes must be 0 (the kernels' count) or 1..1016");
  if (quantum != 0 && quantum != 1 && quantum != 2 && quantum != 4)
    return fail(ILU_EINVAL, "quantum must be 0 (the kernels' own), 1, 2 or 4");
  const int N = 1 << level, q = quantum ? quantum : packed_quantum(N);
  std::string err;
  PackedPlan own;
  const PackedPlan *p = nullptr;
  const int own_lanes = packed_lanes(N);
  if ((lanes == 0 || lanes == own_lanes) && q == packed_quantum(N)) {
    p = packed_plan_cached(N, &err);
  } else if (make_packed_plan(N, lanes ? lanes : own_lanes, q, &own, &err)) {
    p = &own;
  }
  if (!p) return fail(ILU_EINVAL, err);
  *nsteps = p->nsteps;
  *lanes_out = p->lanes;
  const std::vector<PackedEntry> &e = forward ? p->fwd : p->bwd;
  if (entries) std::memcpy(entries, e.data(), sizeof(PackedEntry) * e.size());
  if (lane_off) std::memcpy(lane_off, p->lane_off.data(), sizeof(int) * p->lane_off.size());
  return ILU_OK;
}

ilu_status ilu_profile_enable(ilu_tet t, int enable) {
  ilu::DeviceRestore keep_device;
  if (!t) return fail(ILU_EINVAL, "null handle");
  std::lock_guard<std::mutex> lk(t->mu);
  t->prof = enable != 0;
  return ILU_OK;
}

ilu_status ilu_profile_read(ilu_tet t, double ms[3], long long *launches) {
  ilu::DeviceRestore keep_device;
  if (!t || !ms) return fail(ILU_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(t->mu);
  ms[0] = ms[1] = ms[2] = 0.0;
  if (t->device >= 0) {
    CK(cudaSetDevice(t->device), "cudaSetDevice");
    for (auto &e : t->ev_used) {
      CK(cudaEventSynchronize(e.b), "cudaEventSynchronize");
      float v = 0.f;
      CK(cudaEventElapsedTime(&v, e.a, e.b), "cudaEventElapsedTime");
      if (e.kind >= 0 && e.kind < 3) ms[e.kind] += v;
      t->ev_pool.push_back(e.a);
      t->ev_pool.push_back(e.b);
    }
  }
  t->ev_used.clear();
  if (launches) *launches = t->launches;
  t->launches = 0;
  return ILU_OK;
}

}  // extern "C"
