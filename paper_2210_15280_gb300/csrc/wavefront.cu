// wavefront.cu -- forward and backward substitution of the surrogate ILU(0)
// smoother (arXiv 2210.15280, Alg. 2, V2 boundary rule) on sm_103a.
//
// Level schedule.  Every lower direction d has x+2y+3z weight -1..-3, so the
// points of one hyperplane x + 2y + 3z = s are independent in the forward
// substitution (and, mirrored, in the backward one).  A tet is cut into
// z-slabs; one CTA owns a slab and walks its levels in order.  Each face layer
// of the slab is served by `wpl` compute warps.  In the FP32 sweeps a row
// (y, z) belongs to one lane for its whole life and its polynomials stay in
// registers, evaluated two at a time with packed FMAs; FP64 reads them from
// the shared row cache at every point.
//
// Shared memory per layer:
//   ring   the last 4 levels of w (read by the next three levels),
//   rin    inputs of the next levels (r in the forward pass; the forward
//          result and x in the backward pass), filled by cp.async D levels
//          ahead,
//   coef   the polynomials of every active row, filled by cp.async D levels
//          before the row's first point; in FP64 sweeps with tabulated
//          surrogate values, the 8 values of each point of the next levels
//          instead (filled with the inputs).
// Neighbouring slabs.  The slabs of a tet are launched as thread-block
// clusters.  Inside a cluster the warps of a slab's boundary layer write
// their results straight into the neighbour CTA's halo ring (distributed
// shared memory) and count their arrivals there with a release reduction;
// the neighbour reports its progress back so that a halo slot is never
// overwritten early.  Between clusters a communication warp publishes
// progress in global memory (release, gpu scope) and the receiving one copies
// the boundary layer into its halo ring.  Clusters take numbers from an atomic
// ticket in dependency order, so every wait is on a CTA that is already
// running; every wait is bounded and a timeout sets the status word and ends
// the kernel.
#include <cuda_runtime.h>

#include <climits>

#include "kernels.cuh"

namespace ilu {
namespace {

constexpr int D = 6;    // prefetch distance in levels (inputs, coefficient rows)
constexpr int IS = 8;   // slots of the input rings (> D + 1, power of two)
constexpr int HS = 16;  // slots of the halo ring (power of two)

__device__ __forceinline__ int ylo_of(int N, int s, int z) { return max(1, s - 2 * z - N + 1); }
__device__ __forceinline__ int yhi_of(int N, int s, int z) {
  const int v = s - 3 * z - 1;
  return v < 0 ? 0 : min(v >> 1, N - 2 - z);
}

__device__ __forceinline__ int ld_acq_gpu(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_gpu(int *p, int v) {
  asm volatile("st.release.gpu.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acq_cta(const int *p) {
  int v;
  asm volatile("ld.acquire.cta.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_cta(int *p, int v) {
  asm volatile("st.release.cta.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_rlx_gpu(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// index of (x, y) in face layer z: layer start + row offset + x (32-bit: the
// grid has fewer than 2^31 points up to level 10)
struct LayerIx {
  int start, K1;  // first index of the layer, N - z + 1
  __device__ __forceinline__ int at(int x, int y) const { return start + y * K1 - ((y * (y - 1)) >> 1) + x; }
};
__device__ __forceinline__ LayerIx layer_ix(int N, int z) {
  return LayerIx{(int)layer_start(N, z), N - z + 1};
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

// named barrier over the compute warps; returns the OR of `v` over them
__device__ __forceinline__ bool sync_or(int nthreads, bool v) {
  int out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"((int)v), "r"(nthreads)
      : "memory");
  return out != 0;
}

// Horner evaluation of NF row polynomials (DXP zero-padded coefficients
// each) read from shared memory with 16-byte vector loads.
template <typename T, int DXP, int NF>
__device__ __forceinline__ void eval_rows(const T *c, T t, T (&out)[NF]) {
  constexpr int V = 16 / sizeof(T);
  T a[NF * DXP];
#pragma unroll
  for (int i = 0; i < NF * DXP / V; ++i) {
    if constexpr (sizeof(T) == 4) {
      const float4 q = reinterpret_cast<const float4 *>(c)[i];
      a[4 * i] = q.x; a[4 * i + 1] = q.y; a[4 * i + 2] = q.z; a[4 * i + 3] = q.w;
    } else {
      const double2 q = reinterpret_cast<const double2 *>(c)[i];
      a[2 * i] = q.x; a[2 * i + 1] = q.y;
    }
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    T v = a[f * DXP + DXP - 1];
#pragma unroll
    for (int k = DXP - 2; k >= 0; --k) v = fma(v, t, a[f * DXP + k]);
    out[f] = v;
  }
}

// the 8 tabulated values of one point from shared memory (16-byte loads)
template <typename T>
__device__ __forceinline__ void load_values(const T *v, T (&out)[8]) {
  if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double2 q = reinterpret_cast<const double2 *>(v)[i];
      out[2 * i] = q.x;
      out[2 * i + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = v[i];
  }
}

// two single-precision FMAs in one instruction (fma.rn.f32x2; each lane of
// the pair is an ordinary IEEE fused multiply-add)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  union P {
    float2 f;
    unsigned long long u;
  } A, B, C, R;
  A.f = a;
  B.f = b;
  C.f = c;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(R.u) : "l"(A.u), "l"(B.u), "l"(C.u));
  return R.f;
}

// FP32 row polynomials are stored as four function pairs, coefficient k of
// functions (2p, 2p+1) at float2 index p*DXP + k.  Evaluate all eight from
// shared memory (used when the degree is too high to keep them in registers).
template <int DXP>
__device__ __forceinline__ void eval_pairs_smem(const float *c, float t, float (&out)[8]) {
  const float2 t2 = make_float2(t, t);
  const float2 *q = reinterpret_cast<const float2 *>(c);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    float2 v = q[p * DXP + DXP - 1];
#pragma unroll
    for (int k = DXP - 2; k >= 0; --k) v = ffma2(v, t2, q[p * DXP + k]);
    out[2 * p] = v.x;
    out[2 * p + 1] = v.y;
  }
}

// Coefficients of one row held in registers (degree DX, four function pairs).
template <int DX>
struct RowRegs {
  float2 c[4][DX + 1];
  template <int DXP>
  __device__ __forceinline__ void load(const float *row) {
    const float2 *q = reinterpret_cast<const float2 *>(row);
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int k = 0; k <= DX; ++k) c[p][k] = q[p * DXP + k];
  }
  __device__ __forceinline__ void eval(float t, float (&out)[8]) const {
    const float2 t2 = make_float2(t, t);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float2 v = c[p][DX];
#pragma unroll
      for (int k = DX - 1; k >= 0; --k) v = ffma2(v, t2, c[p][k]);
      out[2 * p] = v.x;
      out[2 * p + 1] = v.y;
    }
  }
};

template <typename T>
__device__ __forceinline__ T *align16(void *p) {
  return reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
}


// ---------------------------------------------------- cluster primitives --

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cl_map(const void *p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_st_int(unsigned a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_st_release(unsigned a, int v) {
  asm volatile("st.release.cluster.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ int cl_ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.cluster.shared::cta.s32 %0, [%1];"
               : "=r"(v)
               : "r"((unsigned)__cvta_generic_to_shared(p))
               : "memory");
  return v;
}
// remote store that completes `sizeof` bytes of a transaction on the remote
// CTA's mbarrier; no fence is involved (the barrier phase orders the data)
__device__ __forceinline__ void cl_st_async(unsigned a, float v, unsigned bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(a), "f"(v), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void cl_st_async(unsigned a, double v, unsigned bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(a), "d"(v), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(b)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"((unsigned)__cvta_generic_to_shared(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// every thread of every CTA of the cluster
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// capacity of the per-layer coefficient cache: the active rows of a level
// (at most N/2) plus the rows fetched ahead
__host__ __device__ __forceinline__ int cache_rows(int N) { return N / 2 + 12; }
// y mod RCC for 1 <= y <= N - 2 < 2 RCC
__device__ __forceinline__ int cache_slot(int y, int RCC) { return y >= RCC ? y - RCC : y; }
// In the register path a cached row is only needed from its fetch, D levels
// before its first point, until its owner lane loads it at that point: a
// ring of kRowRing slots indexed by y mod kRowRing suffices (in either
// direction a row's slot is next refetched at least 10 levels after the load).
constexpr int kRowRing = 16;
template <int REG>
__device__ __forceinline__ int row_slot(int y, int RCC) {
  if constexpr (REG >= 0) return y & (kRowRing - 1);
  else return cache_slot(y, RCC);
}
__host__ __device__ __forceinline__ int level_cap(int N) { return N / 2 + 2; }

// bounded spin of one thread until *p >= target (acquire, cluster scope)
__device__ __forceinline__ bool spin_ge(const int *p, int target, const int *s_abort, long long max_spins) {
  long long spins = 0;
  while (cl_ld_acquire(p) < target) {
    if (*(volatile const int *)s_abort || ++spins > max_spins) return false;
  }
  return true;
}

__device__ __forceinline__ void report_timeout(LaunchStatus *status, int *s_abort, int slab, int level) {
  atomicExch(s_abort, 1);
  if (atomicCAS(&status->code, 0, 6) == 0) {
    status->where = slab;
    status->level = level;
  }
}

// Communication warp.
//   publish: write this slab's progress to global memory (release, gpu scope)
//            for the first slab of the next cluster;
//   listen:  follow the previous cluster's last slab in global memory and copy
//            its boundary layer zh, level by level, into the halo ring;
//   back:    forward this slab's progress to the producing neighbour inside
//            the cluster (its slot guard).
// fwd: progress value = last complete level + 1, levels increase;
// bwd: progress value = TOP - last complete level, levels decrease.
// A halo level v may overwrite slot v % IS once the compute warps have left
// every level that reads the level it replaces.
template <typename TW>
__device__ void comm_warp(bool fwd, int *my_flag, const int *nb_flag, bool publish, bool listen, int back_rank,
                          int *s_done, int *s_nb, int *s_cdone, int *s_abort, int s_begin, int s_end, int N, int zh,
                          int hbase, const TW *wg, TW *halo, int RC, long long max_spins, LaunchStatus *status,
                          int slab) {
  const int lane = threadIdx.x & 31;
  const int TOP = 3 * N + 1;
  const int none = fwd ? INT_MIN : INT_MAX;
  const LayerIx hx = layer_ix(N, zh > 0 ? zh : 1);
  const unsigned back_addr = back_rank >= 0 ? cl_map(s_cdone, (unsigned)back_rank) : 0u;
  int published = 0, nbv = 0, last_done = none, sent = none;
  int next = fwd ? s_begin - 3 : s_end + 3;  // next halo level to fill
  const int last = fwd ? s_end - 1 : s_begin + 1;
  long long idle = 0;
  while (true) {
    const int done = ld_acq_cta(s_done);
    bool prog = done != last_done;
    last_done = done;
    if (done != none && lane == 0) {
      if (publish) {
        const int v = fwd ? done + 1 : TOP - done;
        if (v > published) {
          st_rel_gpu(my_flag, v);
          published = v;
        }
      }
      if (back_rank >= 0 && done != sent) {
        cl_st_release(back_addr, done);
        sent = done;
      }
    }
    if (done == (fwd ? s_end : s_begin)) break;
    if (listen) {
      int v = lane == 0 ? ld_rlx_gpu(nb_flag) : 0;
      v = __shfl_sync(0xffffffffu, v, 0);
      if (v > nbv) {
        fence_gpu();
        nbv = v;
        prog = true;
      }
      const int cdone = done == none ? (fwd ? s_begin - 1 : s_end + 1) : done;
      int filled = 0;
      while (fwd ? (next <= last && next <= nbv - 1 && next <= cdone + HS - 3)
                 : (next >= last && TOP - next <= nbv && next >= cdone - (HS - 3))) {
        const int ylo = ylo_of(N, next, zh), yhi = yhi_of(N, next, zh);
        TW *dst = halo + (size_t)((fwd ? next - hbase : hbase - next) & (HS - 1)) * RC;
        for (int y = ylo + lane; y <= yhi; y += 32) dst[y - ylo] = __ldcg(wg + hx.at(next - 2 * y - 3 * zh, y));
        next += fwd ? 1 : -1;
        ++filled;
      }
      if (filled) {
        __syncwarp();
        if (lane == 0) st_rel_cta(s_nb, fwd ? next : TOP - (next + 1));
        prog = true;
      }
    }
    if (*(volatile int *)s_abort) break;
    if (prog) idle = 0;
    if (++idle > max_spins) {
      if (lane == 0) report_timeout(status, s_abort, slab, done);
      break;
    }
  }
  if (lane == 0) {
    if (publish) st_rel_gpu(my_flag, INT_MAX / 2);  // also releases neighbours after an abort
    if (back_rank >= 0) cl_st_release(back_addr, fwd ? INT_MAX / 2 : INT_MIN / 2);
  }
}

// Halo levels inside a cluster.  The producing CTA stores each point of its
// boundary layer with st.async into the consumer's halo slot and the slot's
// mbarrier counts the bytes.  The consumer arms level v (one arrival plus the
// level's byte count, known from the geometry) and waits for the phase; slot
// and phase come from the position of v in the consumer's sequence of halo
// levels.  `arm` is true for exactly one thread of the CTA.
__device__ __forceinline__ bool wait_halo_level(unsigned long long *hbar, int idx, unsigned bytes, bool arm,
                                                const int *s_abort, long long max_spins) {
  unsigned long long *b = hbar + (idx & (HS - 1));
  if (arm) mbar_arrive_tx(b, bytes);
  const unsigned parity = (unsigned)(idx / HS) & 1u;
  long long spins = 0;
  while (!mbar_test(b, parity)) {
    if (*(volatile const int *)s_abort || ++spins > max_spins) return false;
  }
  return true;
}

// Which tet and which of its clusters a ticket belongs to: the largest j with
// prefix[j] <= ticket (tickets are handed out tet by tet, in bm.order).
__device__ __forceinline__ int ticket_owner(const BatchMap &bm, int ticket) {
  int lo = 0, hi = bm.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bm.prefix[mid] <= ticket) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// --------------------------------------------------------------- forward --

// REG >= 0: FP32 path with the row polynomials (degree REG) in registers,
// each row pinned to one lane for its whole life; REG < 0: polynomials read
// from the shared row cache at every point.
template <typename TW, int DXP, int REG, bool V1>
__global__ void __launch_bounds__(REG >= 0 ? 512 : 1024) fwd_wave(const DevTet *__restrict__ tets, BatchMap bm,
                                                                   LaunchStatus *status, long long max_spins) {
  constexpr int NF = 7;
  constexpr bool F32 = sizeof(TW) == 4;
  constexpr bool TAB = REG == kWaveTabulated;    // values read from t.valsF
  constexpr int ROW = F32 ? 8 * DXP : NF * DXP;  // elements per cached row
  const int NCW = (int)(blockDim.x >> 5) - 1, NCT = NCW * 32;  // compute warps (+ one communication warp)
  __shared__ int s_ticket, s_abort, s_nb, s_done, s_cdone;
  __shared__ __align__(8) unsigned long long hbar[HS];
  const unsigned C = cl_size(), rank = cl_rank();
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_nb = 0;
    s_done = INT_MIN;
    s_cdone = INT_MIN;
    for (int i = 0; i < HS; ++i) mbar_init(&hbar[i], 1);
    mbar_init_fence();
    if (rank == 0) {
      const int tk = atomicAdd(bm.ticket, 1);
      for (unsigned r = 0; r < C; ++r) cl_st_int(cl_map(&s_ticket, r), tk);
    }
  }
  cl_sync();
  const int owner = ticket_owner(bm, s_ticket);
  const DevTet &t = tets[bm.order[owner]];
  const int N = t.N;
  const int Zb = t.fwd.zb, wpl = t.fwd.wpl, P = t.fwd.P;
  const int RC = level_cap(N), RCC = REG >= 0 ? kRowRing : cache_rows(N);
  extern __shared__ __align__(16) unsigned char smem[];
  TW *ring = reinterpret_cast<TW *>(smem);          // [4][Zb][RC]  w of the last levels
  TW *rin = ring + 4 * Zb * RC;                     // [IS][Zb][RC] r of the next levels
  TW *halo = rin + IS * Zb * RC;                    // [HS][RC]     layer z_s - 1
  TW *coef = align16<TW>(halo + HS * RC);           // [Zb][RCC][ROW], tabulated: [IS][Zb][RC][8]
  const int k = (s_ticket - bm.prefix[owner]) * (int)C + (int)rank;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k < P) {
    const int zs = 1 + k * Zb, ze = min(zs + Zb, N - 2);
    const int s_begin = 3 * zs + 3, s_end = 2 * N + ze - 4;
    const bool intra_in = k > 0 && rank > 0;             // halo written by CTA rank-1
    const bool intra_out = k + 1 < P && rank + 1 < C;    // boundary layer goes to CTA rank+1
    TW *wg = reinterpret_cast<TW *>(t.w);
    if (warp == NCW) {
      comm_warp<TW>(true, &t.flags[t.fwd.prog + k], k > 0 ? &t.flags[t.fwd.prog + k - 1] : nullptr,
                    k + 1 < P && rank + 1 == C, k > 0 && rank == 0, intra_in ? (int)rank - 1 : -1, &s_done, &s_nb,
                    &s_cdone, &s_abort, s_begin, s_end, N, zs - 1, 3 * zs, wg, halo, RC, max_spins, status, k);
    } else {
      const int li = warp / wpl, sub = warp - li * wpl;
      const int z = zs + li;
      const bool active = z < ze;
      const bool top = z == ze - 1;
      const TW *tab = reinterpret_cast<const TW *>(t.tabF);
      const TW hh = (TW)(0.5 * t.h);
      const int SS = Zb * RC;
      TW *my_coef = coef + (size_t)li * RCC * ROW;
      const LayerIx ix = layer_ix(N, z);
      const int row0 = active ? (int)row_id(N, 1, z) - 1 : 0;  // row_id(N, y, z) = row0 + y
      const int sb_next = 3 * ze + 3;       // first level of the consuming slab
      const int hlo = 3 * zs;               // first halo level of this slab (layer z_s - 1)
      const int hhi = 2 * N + zs - 4;       // last level of layer z_s - 1
      int hv = hlo;                         // next halo level to wait for
      int cdone_seen = sb_next - 1;         // consumer progress last read (lane 0)

      auto fetch_row = [&](int s2) {  // row of layer z whose first point lies on level s2
        const int v = s2 - 1 - 3 * z;
        if (v < 2 || (v & 1)) return;
        const int y = v >> 1;
        if (y > N - 2 - z) return;
        const char *src = reinterpret_cast<const char *>(tab + (size_t)(row0 + y) * ROW);
        char *dst = reinterpret_cast<char *>(my_coef + (size_t)row_slot<REG>(y, RCC) * ROW);
        constexpr int CH = ROW * (int)sizeof(TW) / 16;
        for (int c = lane; c < CH; c += 32) cp_async<16>(dst + 16 * c, src + 16 * c);
      };
      auto fetch_in = [&](int s2) {  // r (and tabulated values) of this warp's points on level s2
        const int ylo = ylo_of(N, s2, z), yhi = yhi_of(N, s2, z);
        const size_t at = (size_t)(s2 & (IS - 1)) * SS + li * RC;
        for (int y = ylo + 32 * sub + lane; y <= yhi; y += 32 * wpl) {
          const int gi = ix.at(s2 - 2 * y - 3 * z, y);
          cp_async<(int)sizeof(TW)>(rin + at + (y - ylo), wg + gi);
          if constexpr (TAB) {
            const char *src = reinterpret_cast<const char *>(t.valsF + (size_t)gi * 8);
            char *dst = reinterpret_cast<char *>(coef + (at + (y - ylo)) * 8);
#pragma unroll
            for (int c = 0; c < 4; ++c) cp_async<16>(dst + 16 * c, src + 16 * c);
          }
        }
      };

      // register path: the row this lane owns (rows y with (y-1) mod 32*wpl == 32*sub + lane)
      int ycur = 1 + lane + 32 * sub;
      bool have = false;
      RowRegs<(REG >= 0 ? REG : 0)> regs;
      if (active) {
        for (int s2 = s_begin; s2 < s_begin + D; ++s2) {
          if (!TAB && sub == 0) fetch_row(s2);
          fetch_in(s2);
        }
      }
      cp_commit();
      cp_wait<0>();
      bool stop = sync_or(NCT, false);
      for (int s = s_begin; s <= s_end && !stop; ++s) {
        if (active) {
          if (!TAB && sub == 0) fetch_row(s + D);
          fetch_in(s + D);
        }
        cp_commit();
        bool bad = false;
        // layer z_s - 1 on levels up to s - 1 (it has none after 2N + z_s - 4)
        if (active && li == 0 && k > 0) {
          if (intra_in) {
            for (; hv <= min(s - 1, hhi) && !bad; ++hv) {
              const int cnt = max(0, yhi_of(N, hv, zs - 1) - ylo_of(N, hv, zs - 1) + 1);
              bad = !wait_halo_level(hbar, hv - hlo, cnt * (unsigned)sizeof(TW), sub == 0 && lane == 0, &s_abort,
                                     max_spins);
            }
          } else {
            bad = !spin_ge(&s_nb, s, &s_abort, max_spins);
          }
          if (bad && lane == 0) report_timeout(status, &s_abort, k, s);
        }
        // a boundary-layer warp may overwrite the neighbour's halo slot of level
        // s - HS only after the neighbour has left level s - HS + 3
        unsigned hrem = 0, hbar_rem = 0;
        if (top && intra_out && !bad) {
          int ok = 1;
          if (lane == 0 && cdone_seen < s - (HS - 3)) {  // re-read only when the slack is used up
            const int need = s - (HS - 3);
            long long spins = 0;
            while (true) {
              const int c = cl_ld_acquire(&s_cdone);
              cdone_seen = c == INT_MIN ? sb_next - 1 : c;
              if (cdone_seen >= need) break;
              if (*(volatile int *)&s_abort || ++spins > max_spins) {
                ok = 0;
                report_timeout(status, &s_abort, k, s);
                break;
              }
            }
          }
          bad = !__shfl_sync(0xffffffffu, ok, 0);
          const int slot = (s - 3 * ze) & (HS - 1);  // the consumer's halo levels start at 3 z_e
          hrem = cl_map(halo + (size_t)slot * RC, rank + 1);
          hbar_rem = cl_map(&hbar[slot], rank + 1);
        }
        if (active && !bad) {
          const int ylo = ylo_of(N, s, z), yhi = yhi_of(N, s, z);
          const int ylo1 = ylo_of(N, s - 1, z), ylo2 = ylo_of(N, s - 2, z);
          const int zl1 = ylo_of(N, s - 1, z - 1), zl2 = ylo_of(N, s - 2, z - 1), zl3 = ylo_of(N, s - 3, z - 1);
          TW *cur = ring + (size_t)(s & 3) * SS + li * RC;
          const TW *m1 = ring + (size_t)((s - 1) & 3) * SS + li * RC;
          const TW *m2 = ring + (size_t)((s - 2) & 3) * SS + li * RC;
          const TW *b1, *b2, *b3;  // layer z-1 on levels s-1, s-2, s-3
          if (li == 0) {
            b1 = halo + (size_t)((s - 1 - hlo) & (HS - 1)) * RC;
            b2 = halo + (size_t)((s - 2 - hlo) & (HS - 1)) * RC;
            b3 = halo + (size_t)((s - 3 - hlo) & (HS - 1)) * RC;
          } else {
            b1 = m1 - RC;
            b2 = m2 - RC;
            b3 = ring + (size_t)((s - 3) & 3) * SS + (li - 1) * RC;
          }
          const TW *rr = rin + (size_t)(s & (IS - 1)) * SS + li * RC;
          // one point of the forward substitution: L holds L~^p_d, d in D_l
          // boundary variant V1 (instantiated only for launches with such tets)
          const TW *bndv = V1 ? reinterpret_cast<const TW *>(t.bnd) : nullptr;
          auto point = [&](int y, const TW(&Lin)[8]) {
            const int x = s - 2 * y - 3 * z;
            TW L[8];
#pragma unroll
            for (int d = 0; d < 8; ++d) L[d] = Lin[d];
            if constexpr (V1) {
              if (bndv && on_cell_boundary(N, x, y, z)) {  // the stored exact factor at p
                const TW *rec = bndv + (size_t)bnd_record(t.bnd_off, N, x, y, z) * 8;
#pragma unroll
                for (int d = 0; d < 7; ++d) L[d] = rec[d];
              }
            }
            // all operands first, so that their shared-memory latencies
            // overlap; an index outside the row is clamped into it and the
            // value it reads is never used (the V2 tests below skip it)
            auto in = [&](int i) { return min(max(i, 0), RC - 1); };
            const TW vr = rr[y - ylo];
            const TW vw = m1[in(y - ylo1)], vs = m2[in(y - 1 - ylo2)], vse = m1[in(y - 1 - ylo1)];
            TW vbnw = 0, vbn = 0, vbc = 0, vbe = 0;
            if (z >= 2) {  // the same for the whole warp
              vbnw = b2[in(y + 1 - zl2)];
              vbn = b1[in(y + 1 - zl1)];
              vbc = b3[in(y - zl3)];
              vbe = b2[in(y - zl2)];
            }
            TW acc = vr;
            // same layer: w (s-1), s (s-2), se (s-1)
            if (x >= 2) acc = fma(-L[0], vw, acc);
            if (y >= 2) {
              acc = fma(-L[1], vs, acc);
              acc = fma(-L[2], vse, acc);
            }
            // layer below: bnw (s-2), bn (s-1), bc (s-3), be (s-2)
            if (z >= 2) {
              if (x >= 2) acc = fma(-L[3], vbnw, acc);
              acc = fma(-L[4], vbn, acc);
              acc = fma(-L[5], vbc, acc);
              acc = fma(-L[6], vbe, acc);
            }
            cur[y - ylo] = acc;
            if (hrem) cl_st_async(hrem + (unsigned)((y - ylo) * (int)sizeof(TW)), acc, hbar_rem);
            wg[ix.at(x, y)] = acc;
          };
          if constexpr (REG >= 0) {
            while (ycur < ylo) {
              ycur += 32 * wpl;
              have = false;
            }
            if (ycur <= yhi) {
              if (!have) {
                regs.template load<DXP>(reinterpret_cast<const float *>(my_coef) + (size_t)row_slot<REG>(ycur, RCC) * ROW);
                have = true;
              }
              const int x = s - 2 * ycur - 3 * z;
              TW L[8];
              regs.eval((TW)(2 * x - (N - ycur - z)) * hh, L);
              point(ycur, L);
            }
          } else if constexpr (TAB) {
            const TW *vv = coef + ((size_t)(s & (IS - 1)) * SS + li * RC) * 8;
            for (int y = ylo + 32 * sub + lane; y <= yhi; y += 32 * wpl) {
              TW L[8];
              load_values(vv + (size_t)(y - ylo) * 8, L);
              point(y, L);
            }
          } else {
            int slot = ylo % RCC + 32 * sub + lane;
            for (int y = ylo + 32 * sub + lane; y <= yhi; y += 32 * wpl, slot += 32 * wpl) {
              if (slot >= RCC) slot -= RCC;
              const int x = s - 2 * y - 3 * z;
              const TW tt = (TW)(2 * x - (N - y - z)) * hh;
              TW L[8];
              if constexpr (F32) {
                eval_pairs_smem<DXP>(reinterpret_cast<const float *>(my_coef) + (size_t)slot * ROW, (float)tt,
                                     reinterpret_cast<float(&)[8]>(L));
              } else {
                TW L7[NF];
                eval_rows<TW, DXP, NF>(my_coef + (size_t)slot * ROW, tt, L7);
#pragma unroll
                for (int f = 0; f < NF; ++f) L[f] = L7[f];
              }
              point(y, L);
            }
          }
        }
        cp_wait<D - 1>();
        stop = sync_or(NCT, bad || *(volatile int *)&s_abort);
        if (threadIdx.x == 0) st_rel_cta(&s_done, s);
      }
      cp_wait<0>();
      if (threadIdx.x == 0 && stop) atomicExch(&s_abort, 1);
    }
  }
  cl_sync();  // no CTA leaves while a neighbour may still write into its shared memory
}

// -------------------------------------------------------------- backward --

template <typename TW, typename TX, int DXP, int REG, bool V1>
__global__ void __launch_bounds__(REG >= 0 ? 512 : 1024) bwd_wave(const DevTet *__restrict__ tets, BatchMap bm,
                                                                   LaunchStatus *status, long long max_spins) {
  constexpr int NF = 8;
  constexpr bool F32 = sizeof(TW) == 4;
  constexpr bool TAB = REG == kWaveTabulated;  // values read from t.valsB
  constexpr int ROW = NF * DXP;  // elements per cached row (FP32: 4 pairs x DXP x 2)
  const int NCW = (int)(blockDim.x >> 5) - 1, NCT = NCW * 32;
  __shared__ int s_ticket, s_abort, s_nb, s_done, s_cdone;
  __shared__ __align__(8) unsigned long long hbar[HS];
  const unsigned C = cl_size(), rank = cl_rank();
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_nb = 0;
    s_done = INT_MAX;
    s_cdone = INT_MAX;
    for (int i = 0; i < HS; ++i) mbar_init(&hbar[i], 1);
    mbar_init_fence();
    if (rank == 0) {
      const int tk = atomicAdd(bm.ticket, 1);
      for (unsigned r = 0; r < C; ++r) cl_st_int(cl_map(&s_ticket, r), tk);
    }
  }
  cl_sync();
  const int owner = ticket_owner(bm, s_ticket);
  const int ti = bm.order[owner];
  const DevTet &t = tets[ti];
  TX *__restrict__ xg = reinterpret_cast<TX *>(bm.xs ? bm.xs[ti] : bm.x0);
  const int N = t.N;
  const int Zb = t.bwd.zb, wpl = t.bwd.wpl, P = t.bwd.P;
  const int RC = level_cap(N), RCC = REG >= 0 ? kRowRing : cache_rows(N);
  const int TOP = 3 * N + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  TW *ring = reinterpret_cast<TW *>(smem);       // [4][Zb][RC]
  TW *win = ring + 4 * Zb * RC;                  // [IS][Zb][RC] forward result of the next levels
  TW *halo = win + IS * Zb * RC;                 // [HS][RC]     layer z_e
  TX *xin = align16<TX>(halo + HS * RC);         // [IS][Zb][RC] x of the next levels
  TW *coef = align16<TW>(xin + IS * Zb * RC);    // [Zb][RCC][ROW], tabulated: [IS][Zb][RC][8]
  const int Q = bm.prefix[owner + 1] - bm.prefix[owner];  // clusters of this tet
  const int k = (Q - 1 - (s_ticket - bm.prefix[owner])) * (int)C + (int)rank;  // top clusters first
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k < P) {
    const int zs = 1 + k * Zb, ze = min(zs + Zb, N - 2);
    const int s_begin = 3 * zs + 3, s_end = 2 * N + ze - 4;
    const bool intra_in = k + 1 < P && rank + 1 < C;  // halo written by CTA rank+1
    const bool intra_out = k > 0 && rank > 0;         // bottom layer goes to CTA rank-1
    TW *wg = reinterpret_cast<TW *>(t.w);
    if (warp == NCW) {
      comm_warp<TW>(false, &t.flags[t.bwd.prog + k], k + 1 < P ? &t.flags[t.bwd.prog + k + 1] : nullptr,
                    k > 0 && rank == 0, k + 1 < P && rank + 1 == C, intra_in ? (int)rank + 1 : -1, &s_done, &s_nb,
                    &s_cdone, &s_abort, s_begin, s_end, N, ze, 2 * N + ze - 3, wg, halo, RC, max_spins, status, k);
    } else {
      const int li = warp / wpl, sub = warp - li * wpl;
      const int z = zs + li;
      const bool active = z < ze;
      const bool top = z + 1 >= ze;  // layer z+1 belongs to the slab above
      const bool bottom = li == 0;
      const TW *tab = reinterpret_cast<const TW *>(t.tabB);
      const TW hh = (TW)(0.5 * t.h);
      const int SS = Zb * RC;
      TW *my_coef = coef + (size_t)li * RCC * ROW;
      const LayerIx ix = layer_ix(N, z);
      const int row0 = active ? (int)row_id(N, 1, z) - 1 : 0;  // row_id(N, y, z) = row0 + y
      const int se_next = 2 * N + zs - 4;  // first level of the consuming slab below
      const int hhi = 2 * N + ze - 3;      // first halo level of this slab (layer z_e, descending)
      const int hlo = 3 * ze + 3;          // last level of layer z_e
      int hv = hhi;                        // next halo level to wait for
      int cdone_seen = se_next + 1;        // consumer progress last read (lane 0)

      auto fetch_row = [&](int s2) {  // row of layer z whose last point lies on level s2
        const int y = s2 - (N - 1) - 2 * z;
        if (y < 1 || y > N - 2 - z) return;
        const char *src = reinterpret_cast<const char *>(tab + (size_t)(row0 + y) * ROW);
        char *dst = reinterpret_cast<char *>(my_coef + (size_t)row_slot<REG>(y, RCC) * ROW);
        constexpr int CH = ROW * (int)sizeof(TW) / 16;
        for (int c = lane; c < CH; c += 32) cp_async<16>(dst + 16 * c, src + 16 * c);
      };
      auto fetch_in = [&](int s2) {  // forward result, x (and tabulated values) of this warp's points on level s2
        const int ylo = ylo_of(N, s2, z), yhi = yhi_of(N, s2, z);
        const size_t at = (size_t)(s2 & (IS - 1)) * SS + li * RC;
        for (int y = ylo + 32 * sub + lane; y <= yhi; y += 32 * wpl) {
          const int gi = ix.at(s2 - 2 * y - 3 * z, y);
          cp_async<(int)sizeof(TW)>(win + at + (y - ylo), wg + gi);
          cp_async<(int)sizeof(TX)>(xin + at + (y - ylo), xg + gi);
          if constexpr (TAB) {
            const char *src = reinterpret_cast<const char *>(t.valsB + (size_t)gi * 8);
            char *dst = reinterpret_cast<char *>(coef + (at + (y - ylo)) * 8);
#pragma unroll
            for (int c = 0; c < 4; ++c) cp_async<16>(dst + 16 * c, src + 16 * c);
          }
        }
      };

      // register path: the highest row this lane owns, walked downwards
      int ycur = 1 + lane + 32 * sub;
      if (ycur <= N - 2 - z) ycur += ((N - 2 - z - ycur) / (32 * wpl)) * (32 * wpl);
      bool have = false;
      RowRegs<(REG >= 0 ? REG : 0)> regs;
      if (active) {
        for (int s2 = s_end; s2 > s_end - D; --s2) {
          if (!TAB && sub == 0) fetch_row(s2);
          fetch_in(s2);
        }
      }
      cp_commit();
      cp_wait<0>();
      bool stop = sync_or(NCT, false);
      for (int s = s_end; s >= s_begin && !stop; --s) {
        if (active) {
          if (!TAB && sub == 0) fetch_row(s - D);
          fetch_in(s - D);
        }
        cp_commit();
        bool bad = false;
        // layer z_e on levels down to s + 1 (it has none below 3 z_e + 3)
        if (active && top && k + 1 < P) {
          if (intra_in) {
            for (; hv >= max(s + 1, hlo) && !bad; --hv) {
              const int cnt = max(0, yhi_of(N, hv, ze) - ylo_of(N, hv, ze) + 1);
              bad = !wait_halo_level(hbar, hhi - hv, cnt * (unsigned)sizeof(TW), sub == 0 && lane == 0, &s_abort,
                                     max_spins);
            }
          } else {
            bad = !spin_ge(&s_nb, TOP - (s + 1), &s_abort, max_spins);
          }
          if (bad && lane == 0) report_timeout(status, &s_abort, k, s);
        }
        unsigned hrem = 0, hbar_rem = 0;
        if (bottom && intra_out && !bad) {
          int ok = 1;
          if (lane == 0 && cdone_seen > s + (HS - 3)) {  // re-read only when the slack is used up
            const int need = s + (HS - 3);
            long long spins = 0;
            while (true) {
              const int c = cl_ld_acquire(&s_cdone);
              cdone_seen = c == INT_MAX ? se_next + 1 : c;
              if (cdone_seen <= need) break;
              if (*(volatile int *)&s_abort || ++spins > max_spins) {
                ok = 0;
                report_timeout(status, &s_abort, k, s);
                break;
              }
            }
          }
          bad = !__shfl_sync(0xffffffffu, ok, 0);
          const int slot = (2 * N + zs - 3 - s) & (HS - 1);  // the consumer's halo levels start at 2N + z_s - 3
          hrem = cl_map(halo + (size_t)slot * RC, rank - 1);
          hbar_rem = cl_map(&hbar[slot], rank - 1);
        }
        if (active && !bad) {
          const int ylo = ylo_of(N, s, z), yhi = yhi_of(N, s, z);
          const int ylo1 = ylo_of(N, s + 1, z), ylo2 = ylo_of(N, s + 2, z);
          const int zl1 = ylo_of(N, s + 1, z + 1), zl2 = ylo_of(N, s + 2, z + 1), zl3 = ylo_of(N, s + 3, z + 1);
          TW *cur = ring + (size_t)(s & 3) * SS + li * RC;
          const TW *p1 = ring + (size_t)((s + 1) & 3) * SS + li * RC;
          const TW *p2 = ring + (size_t)((s + 2) & 3) * SS + li * RC;
          const TW *u1, *u2, *u3;  // layer z+1 on levels s+1, s+2, s+3
          if (top) {
            u1 = halo + (size_t)((hhi - s - 1) & (HS - 1)) * RC;
            u2 = halo + (size_t)((hhi - s - 2) & (HS - 1)) * RC;
            u3 = halo + (size_t)((hhi - s - 3) & (HS - 1)) * RC;
          } else {
            u1 = p1 + RC;
            u2 = p2 + RC;
            u3 = ring + (size_t)((s + 3) & 3) * SS + (li + 1) * RC;
          }
          const TW *ww = win + (size_t)(s & (IS - 1)) * SS + li * RC;
          const TX *xx = xin + (size_t)(s & (IS - 1)) * SS + li * RC;
          const bool store_w = bottom && k > 0 && !intra_out;  // the next cluster reads this layer
          // one point of the backward substitution: L[0] = 1/D~^p, L[1+d] = L~^{p-d}_d
          const TW *bndv = V1 ? reinterpret_cast<const TW *>(t.bnd) : nullptr;
          auto point = [&](int y, const TW(&Lin)[8]) {
            const int x = s - 2 * y - 3 * z;
            TW L[8];
#pragma unroll
            for (int d = 0; d < 8; ++d) L[d] = Lin[d];
            if (V1 && bndv) {  // L~^{p-d}_d from the stored exact factor where p - d is on the cell boundary
              if (on_cell_boundary(N, x, y, z)) L[0] = bndv[(size_t)bnd_record(t.bnd_off, N, x, y, z) * 8 + 7];
#pragma unroll
              for (int d = 0; d < kNumLower; ++d) {
                const int qx = x - dir_dx(d), qy = y - dir_dy(d), qz = z - dir_dz(d);
                if (in_interior(N, qx, qy, qz) && on_cell_boundary(N, qx, qy, qz))
                  L[1 + d] = bndv[(size_t)bnd_record(t.bnd_off, N, qx, qy, qz) * 8 + d];
              }
            }
            // operands first (clamped indices, as in the forward kernel)
            auto in = [&](int i) { return min(max(i, 0), RC - 1); };
            const TW vw0 = ww[y - ylo];
            const TW vw = p1[in(y - ylo1)], vs = p2[in(y + 1 - ylo2)], vbc = u3[in(y - zl3)];
            const TW vbnw = u2[in(y - 1 - zl2)], vse = p1[in(y + 1 - ylo1)], vbe = u2[in(y - zl2)];
            const TW vbn = u1[in(y - 1 - zl1)];
            TW acc = L[0] * vw0;
            const bool inner = x + y + z <= N - 2;  // p - w, p - s, p - bc interior
            if (inner) {
              acc = fma(-L[1], vw, acc);   // p - w  = (x+1, y, z)
              acc = fma(-L[2], vs, acc);   // p - s  = (x, y+1, z)
              acc = fma(-L[6], vbc, acc);  // p - bc = (x, y, z+1)
              if (y >= 2) acc = fma(-L[4], vbnw, acc);  // p - bnw = (x+1, y-1, z+1)
            }
            if (x >= 2) {
              acc = fma(-L[3], vse, acc);  // p - se = (x-1, y+1, z)
              acc = fma(-L[7], vbe, acc);  // p - be = (x-1, y, z+1)
            }
            if (y >= 2) acc = fma(-L[5], vbn, acc);  // p - bn = (x, y-1, z+1)
            cur[y - ylo] = acc;
            if (hrem) cl_st_async(hrem + (unsigned)((y - ylo) * (int)sizeof(TW)), acc, hbar_rem);
            const int gi = ix.at(x, y);
            if (store_w) wg[gi] = acc;
            xg[gi] = xx[y - ylo] + (TX)acc;
          };
          if constexpr (REG >= 0) {
            while (ycur > yhi) {
              ycur -= 32 * wpl;
              have = false;
            }
            if (ycur >= ylo) {
              if (!have) {
                regs.template load<DXP>(reinterpret_cast<const float *>(my_coef) + (size_t)row_slot<REG>(ycur, RCC) * ROW);
                have = true;
              }
              const int x = s - 2 * ycur - 3 * z;
              TW L[8];
              regs.eval((TW)(2 * x - (N - ycur - z)) * hh, L);
              point(ycur, L);
            }
          } else if constexpr (TAB) {
            const TW *vv = coef + ((size_t)(s & (IS - 1)) * SS + li * RC) * 8;
            for (int y = ylo + 32 * sub + lane; y <= yhi; y += 32 * wpl) {
              TW L[8];
              load_values(vv + (size_t)(y - ylo) * 8, L);
              point(y, L);
            }
          } else {
            int slot = ylo % RCC + 32 * sub + lane;
            for (int y = ylo + 32 * sub + lane; y <= yhi; y += 32 * wpl, slot += 32 * wpl) {
              if (slot >= RCC) slot -= RCC;
              const int x = s - 2 * y - 3 * z;
              const TW tt = (TW)(2 * x - (N - y - z)) * hh;
              TW L[8];
              if constexpr (F32)
                eval_pairs_smem<DXP>(reinterpret_cast<const float *>(my_coef) + (size_t)slot * ROW, (float)tt,
                                     reinterpret_cast<float(&)[8]>(L));
              else
                eval_rows<TW, DXP, NF>(my_coef + (size_t)slot * ROW, tt, L);
              point(y, L);
            }
          }
        }
        cp_wait<D - 1>();
        stop = sync_or(NCT, bad || *(volatile int *)&s_abort);
        if (threadIdx.x == 0) st_rel_cta(&s_done, s);
      }
      cp_wait<0>();
      if (threadIdx.x == 0 && stop) atomicExch(&s_abort, 1);
    }
  }
  cl_sync();
}

// coefficient area: row polynomials (register ring or row cache), or the
// tabulated values of the next IS levels
template <typename TW>
size_t coef_smem(int N, const WaveGeom &g, int dxp, int reg, int nf) {
  const size_t RC = level_cap(N);
  if (reg == kWaveTabulated) return sizeof(TW) * IS * g.zb * RC * 8;
  const size_t RCC = reg >= 0 ? kRowRing : cache_rows(N);
  return (size_t)g.zb * RCC * nf * dxp * sizeof(TW);
}
template <typename TW>
size_t fwd_smem(int N, const WaveGeom &g, int dxp, int reg) {
  const size_t RC = level_cap(N);
  return sizeof(TW) * ((4 + IS) * g.zb * RC + HS * RC) + 16 + coef_smem<TW>(N, g, dxp, reg, sizeof(TW) == 4 ? 8 : 7);
}
template <typename TW, typename TX>
size_t bwd_smem(int N, const WaveGeom &g, int dxp, int reg) {
  const size_t RC = level_cap(N);
  return sizeof(TW) * ((4 + IS) * g.zb * RC + HS * RC) + 16 + sizeof(TX) * IS * g.zb * RC + 16 +
         coef_smem<TW>(N, g, dxp, reg, 8);
}

// Launch as clusters of `csize` CTAs covering `clusters` clusters.  With
// `query` set nothing is launched (see launch_forward).
template <typename K>
cudaError_t cluster_launch(K kernel, const WaveLaunch &L, bool fwd, cudaStream_t st, int *query, LaunchStatus *status,
                           long long max_spins) {
  const size_t smem = fwd ? L.smem_f : L.smem_b;
  // The dynamic shared-memory cap is a property of the kernel, shared by
  // every thread and launch in the process: raise it to the device's opt-in
  // limit less the kernel's static shared memory (the same value from every
  // caller) rather than to this launch's need, which would race with
  // concurrent launches of other tets.
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int cap = optin - (int)fa.sharedSizeBytes;
  if (smem > (size_t)cap) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(fwd ? L.block_f : L.block_b);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query) {
    const int maxP = fwd ? L.maxP_f : L.maxP_b;
    query[0] = 1;
    bool found = false;
    for (int i = 0; i < kClusterCands; ++i) {
      const int cs = kClusterSizes[i] < maxP ? kClusterSizes[i] : maxP;
      attr[0].val.clusterDim.x = cs;
      cfg.gridDim = dim3(cs);
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
      }
      query[1 + i] = n;
      if (n > 0 && !found) {
        query[0] = cs;
        found = true;
      }
    }
    return cudaSuccess;
  }
  const int cs = fwd ? L.csize_f : L.csize_b;
  attr[0].val.clusterDim.x = cs;
  cfg.gridDim = dim3((fwd ? L.clusters_f : L.clusters_b) * cs);
  return cudaLaunchKernelEx(&cfg, kernel, L.tets, fwd ? L.map_f : L.map_b, status, max_spins);
}

template <typename TW, int DXP, int REG>
cudaError_t fwd_launch(const WaveLaunch &L, LaunchStatus *status, long long max_spins, cudaStream_t st, int *query) {
  if (L.v1) return cluster_launch(fwd_wave<TW, DXP, REG, true>, L, true, st, query, status, max_spins);
  return cluster_launch(fwd_wave<TW, DXP, REG, false>, L, true, st, query, status, max_spins);
}

template <typename TW, typename TX, int DXP, int REG>
cudaError_t bwd_launch(const WaveLaunch &L, LaunchStatus *status, long long max_spins, cudaStream_t st, int *query) {
  if (L.v1) return cluster_launch(bwd_wave<TW, TX, DXP, REG, true>, L, false, st, query, status, max_spins);
  return cluster_launch(bwd_wave<TW, TX, DXP, REG, false>, L, false, st, query, status, max_spins);
}

// FP32 dispatch on the register degree; rows of degree <= 3 are stored with
// 4 coefficients per function, degree 4..7 with 8
cudaError_t fwd32(const WaveLaunch &L, LaunchStatus *s, long long m, cudaStream_t st, int *q) {
  switch (L.reg) {
    case 0: return fwd_launch<float, 4, 0>(L, s, m, st, q);
    case 1: return fwd_launch<float, 4, 1>(L, s, m, st, q);
    case 2: return fwd_launch<float, 4, 2>(L, s, m, st, q);
    case 3: return fwd_launch<float, 4, 3>(L, s, m, st, q);
    case 4: return fwd_launch<float, 8, 4>(L, s, m, st, q);
    case 5: return fwd_launch<float, 8, 5>(L, s, m, st, q);
    case 6: return fwd_launch<float, 8, 6>(L, s, m, st, q);
    case 7: return fwd_launch<float, 8, 7>(L, s, m, st, q);
    default: return fwd_launch<float, 16, -1>(L, s, m, st, q);
  }
}
template <typename TX>
cudaError_t bwd32(const WaveLaunch &L, LaunchStatus *s, long long m, cudaStream_t st, int *q) {
  switch (L.reg) {
    case 0: return bwd_launch<float, TX, 4, 0>(L, s, m, st, q);
    case 1: return bwd_launch<float, TX, 4, 1>(L, s, m, st, q);
    case 2: return bwd_launch<float, TX, 4, 2>(L, s, m, st, q);
    case 3: return bwd_launch<float, TX, 4, 3>(L, s, m, st, q);
    case 4: return bwd_launch<float, TX, 8, 4>(L, s, m, st, q);
    case 5: return bwd_launch<float, TX, 8, 5>(L, s, m, st, q);
    case 6: return bwd_launch<float, TX, 8, 6>(L, s, m, st, q);
    case 7: return bwd_launch<float, TX, 8, 7>(L, s, m, st, q);
    default: return bwd_launch<float, TX, 16, -1>(L, s, m, st, q);
  }
}

// Surrogate values of every interior point for FP64 sweeps that read them
// from tables: one block per row (y, z), threads over x.  The values are the
// ones the substitutions would evaluate themselves: the same row
// polynomials, the same abscissa and the same Horner steps (eval_rows), so
// the two ways give bit-identical sweeps.
template <int DXP>
__global__ void __launch_bounds__(128) tabulate_kernel(const DevTet t, double *__restrict__ valsF,
                                                       double *__restrict__ valsB) {
  const int N = t.N;
  const int y = (int)blockIdx.x + 1, z = (int)blockIdx.y + 1;
  if (y > N - 2 - z) return;
  const LayerIx ix = layer_ix(N, z);
  const size_t row = (size_t)row_id(N, y, z);
  const double *cf = reinterpret_cast<const double *>(t.tabF) + row * 7 * DXP;
  const double *cb = reinterpret_cast<const double *>(t.tabB) + row * 8 * DXP;
  const double hh = (double)(0.5 * t.h);
  for (int x = 1 + (int)threadIdx.x; x <= N - 1 - y - z; x += (int)blockDim.x) {
    const double tt = (double)(2 * x - (N - y - z)) * hh;
    double f[7], b[8];
    eval_rows<double, DXP, 7>(cf, tt, f);
    eval_rows<double, DXP, 8>(cb, tt, b);
    const size_t gi = (size_t)ix.at(x, y);
    double2 *of = reinterpret_cast<double2 *>(valsF + gi * 8);
    double2 *ob = reinterpret_cast<double2 *>(valsB + gi * 8);
    of[0] = make_double2(f[0], f[1]);
    of[1] = make_double2(f[2], f[3]);
    of[2] = make_double2(f[4], f[5]);
    of[3] = make_double2(f[6], 0.0);
#pragma unroll
    for (int i = 0; i < 4; ++i) ob[i] = make_double2(b[2 * i], b[2 * i + 1]);
  }
}

}  // namespace

cudaError_t launch_tabulate(const DevTet &t, double *valsF, double *valsB, cudaStream_t st) {
  if (t.N < 4) return cudaSuccess;
  const dim3 grid(t.N - 3, t.N - 3);
  switch (t.rstride) {
    case 4: tabulate_kernel<4><<<grid, 128, 0, st>>>(t, valsF, valsB); break;
    case 8: tabulate_kernel<8><<<grid, 128, 0, st>>>(t, valsF, valsB); break;
    case 16: tabulate_kernel<16><<<grid, 128, 0, st>>>(t, valsF, valsB); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

bool wave_uses_registers(int kind, int dx) { return kind != kSweepF64 && dx <= 7; }

size_t wave_smem_bytes(int N, const WaveGeom &g, int kind, int dxp, int reg, bool forward) {
  if (forward) return kind == kSweepF64 ? fwd_smem<double>(N, g, dxp, reg) : fwd_smem<float>(N, g, dxp, reg);
  if (kind == kSweepF64) return bwd_smem<double, double>(N, g, dxp, reg);
  if (kind == kSweepMixed) return bwd_smem<float, double>(N, g, dxp, reg);
  return bwd_smem<float, float>(N, g, dxp, reg);
}

cudaError_t launch_forward(const WaveLaunch &L, LaunchStatus *status, long long max_spins, cudaStream_t st,
                           int *cluster_query) {
  if (L.kind == kSweepF64) {
    if (L.reg == kWaveTabulated) return fwd_launch<double, 4, kWaveTabulated>(L, status, max_spins, st, cluster_query);
    if (L.dxp == 4) return fwd_launch<double, 4, -1>(L, status, max_spins, st, cluster_query);
    if (L.dxp == 8) return fwd_launch<double, 8, -1>(L, status, max_spins, st, cluster_query);
    return fwd_launch<double, 16, -1>(L, status, max_spins, st, cluster_query);
  }
  return fwd32(L, status, max_spins, st, cluster_query);
}

cudaError_t launch_backward(const WaveLaunch &L, LaunchStatus *status, long long max_spins, cudaStream_t st,
                            int *cluster_query) {
  if (L.kind == kSweepF64) {
    if (L.reg == kWaveTabulated)
      return bwd_launch<double, double, 4, kWaveTabulated>(L, status, max_spins, st, cluster_query);
    if (L.dxp == 4) return bwd_launch<double, double, 4, -1>(L, status, max_spins, st, cluster_query);
    if (L.dxp == 8) return bwd_launch<double, double, 8, -1>(L, status, max_spins, st, cluster_query);
    return bwd_launch<double, double, 16, -1>(L, status, max_spins, st, cluster_query);
  }
  if (L.kind == kSweepMixed) return bwd32<double>(L, status, max_spins, st, cluster_query);
  return bwd32<float>(L, status, max_spins, st, cluster_query);
}

}  // namespace ilu
