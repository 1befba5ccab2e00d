// packed.cu -- packed substitution kernels of the FP32 sweeps (Alg. 2 of
// arXiv 2210.15280 with the V2 boundary rule; V1 as an option).
//
// One CTA of kPackedLanes threads per macro-tetrahedron (at level 8 a
// cluster of two CTAs of kPackedClusterLanes threads, each holding the
// whole ring) runs the forward substitution
//     w^p = r^p - sum_{d in D_l, p+d interior} L~^p_d w^{p+d}
// and then the backward substitution
//     w^p <- D~^-1(p) w^p - sum_{d in D_l, p-d interior} L~^{p-d}_d w^{p-d},
// walking the steps of the tet's host-computed row schedule (packed.h): at
// step tau every lane computes one point of the row it owns (or writes 0),
// and every Q steps the CTA (cluster) meets at a barrier.  No tet waits on
// another.  Everything the
// passes read and write lies in the tet's step-major packed array, where the
// lanes of a warp touch consecutive words at every step; packed_io_kernel
// moves vectors between the lexicographic grid and that array (the residual
// kernel writes r there directly).
//
// Per lane:
//   registers  the row polynomials of its current row (four function pairs,
//              evaluated two at a time by packed FMAs), the previous value of
//              its own row, the producer values carried from the last step;
//   ring       its results of the last kPackedRing steps (shared memory);
//              consumers read producer values there by (step, lane);
//   queue      the values of producer rows that ran too far ahead for the
//              ring, read back from the packed array kPackedPre steps ahead
//              -- filled by cp.async;
//   stage      the next row's coefficients and the schedule entry after it,
//              filled by cp.async while the current row runs.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "kernels.cuh"
#include "packed.h"

namespace ilu {
namespace {

constexpr int RG = kPackedRing, QS = kPackedQueue, PD = kPackedPre;
constexpr int RR = RG + kPackedBlock;      // ring rows: RG, then a mirror of rows 0 .. kPackedBlock - 1
// threads per CTA, and words per ring row (all lanes of the tet's CTA or
// cluster, then 8 words; column CL * cta_lanes(CL) is never written: reads 0)
__host__ __device__ constexpr int cta_lanes(int cl) { return cl > 1 ? kPackedClusterLanes : kPackedLanes; }
__host__ __device__ constexpr int ring_row(int cl) { return packed_ring_row(cl * cta_lanes(cl)); }
static_assert((RG & (RG - 1)) == 0 && (QS & (QS - 1)) == 0, "ring and queue sizes are powers of two");
static_assert(QS == kPackedBlock, "a step's queue slot is its index in the unrolled block");
static_assert(RG % kPackedBlock == 0, "blocks tile the ring");
static_assert(PD < QS, "the entry read at a step must not be the one being refilled");
static_assert(RG - 1 >= PD + 1, "ring and global reads must cover every producer distance");

template <int BYTES>
__device__ __forceinline__ void cpa(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src),
               "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cpa16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  union U {
    float2 f;
    unsigned long long u;
  } A, B, C, R;
  A.f = a;
  B.f = b;
  C.f = c;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(R.u) : "l"(A.u), "l"(B.u), "l"(C.u));
  return R.f;
}

__device__ __forceinline__ int pmode(int code) { return (code >> 30) & 3; }

// cluster primitives: this CTA's rank, the cluster-window address of a
// shared location in CTA `rank`, a store through that window, and a barrier
// of every thread of the cluster (release / acquire: shared-memory writes
// before it, the other CTA's included, are visible to every CTA after it)
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_addr(const void *p, unsigned rank) {
  unsigned a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(rank));
  return a;
}
__device__ __forceinline__ void st_cluster(unsigned a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the barrier of a packed pass: the CTA's, or the cluster's for CL > 1
template <int CL>
__device__ __forceinline__ void pass_sync() {
  if constexpr (CL > 1) cluster_sync_all();
  else __syncthreads();
}

// One substitution of one tet on one CTA.
//
// Lane state: the current row (its points' steps [lo, lo + n), the ring word
// of each producer's read at the current block's first step, which
// producers come through the queue), the value each producer gave at the
// last step (a consumer's first value at a step is its second value of the
// step before, so one read per producer and step suffices), the lane's own
// value of the last step, the row coordinate t of the step's point (advanced
// by h per step; every value is a small dyadic fraction, so the sums are
// exact), and the next row's schedule entry.  Two per-lane events change it:
// kPackedPre steps before the next row's switch step the prefetch cursor
// moves to that row and the copies of its coefficients and of the entry
// after it are issued; on the switch step the row becomes current
// (coefficients from the stage, the entry after it from `sent`).  Switch
// steps are Q - 1 (mod Q), so only those unrolled positions test for events.
//
// The CTA (cluster) meets at a barrier after every step Q - 1 (mod Q): the
// schedule keeps every producer value at least Q + 1 steps ahead of the step
// that reads it and reads the ring only up to kPackedRing + 1 - Q steps back,
// so a value is visible when read and not yet overwritten, however far apart
// the lanes are between two barriers.  In a cluster each CTA holds the ring
// of all lanes: a lane writes its result into its own CTA's ring and the
// other's, and the barrier's release and acquire order both.  A lane's own stage and `sent` are
// refilled only after the barrier that follows the switch step reading them.
//
// Steps with no point of the lane write 0.  The schedule leaves such a step
// before and after every row, in both passes, and these are exactly the
// steps at which a consumer reads a producer's missing neighbour (x = 0, or
// one past the producer row's end); a producer row that does not exist is
// read from ring column LT (after every lane's column), which is never
// written.  So the point arithmetic needs no masks.
//
// The loop runs in blocks of kPackedBlock steps, unrolled, so that ring rows
// and queue slots are compile-time offsets from per-block bases: ring row
// (tau & (RG-1)) holds step tau's results, and the first kPackedBlock rows
// are mirrored after row RG - 1 so that a producer's reads within a block
// never wrap.  Inputs are read and results written four steps at a time (one
// 16-byte block per lane).
template <bool FWD, int DX, bool V1, int Q, int CL>
__device__ __forceinline__ void packed_pass(const DevTet &t, unsigned char *smem) {
  constexpr int SF2 = 4 * (DX + 1);  // float2 of a staged row: coefficient k of the four function pairs
  constexpr int LN = cta_lanes(CL);  // this CTA's lanes
  constexpr int LT = CL * LN;        // lanes of the schedule and the packed array
  constexpr int RW = ring_row(CL);
  float *ring = reinterpret_cast<float *>(smem);                 // [RR][RW]
  float4 *q = reinterpret_cast<float4 *>(ring + RR * RW);        // [QS][LN] far producer values (.y .z .w)
  int4 *sent = reinterpret_cast<int4 *>(q + QS * LN);            // [LN][2]
  float2 *stage = reinterpret_cast<float2 *>(sent + 2 * LN);     // [LN][SF2]
  const int lane = threadIdx.x;                                    // this CTA's lane (stage, sent)
  const unsigned rank = CL > 1 ? cluster_rank() : 0u;
  const int lg = (int)rank * LN + lane;                            // the schedule's lane (ring column)
  const int N = t.N;
  const int4 *ent = FWD ? t.pk.ent_f : t.pk.ent_b;  // entry e at ent[2e], ent[2e + 1]
  const int *off = t.pk.off;
  const int T = t.pk.nsteps;  // a multiple of kPackedBlock
  const float2 *tab = reinterpret_cast<const float2 *>(FWD ? t.pkF : t.pkB);
  float *pw = t.pk.pw;  // packed array; backward step tau works on forward step T - 1 - tau
  const float hh = (float)(0.5 * t.h);
  float2 *my_stage = stage + lane * SF2;

  // ring rows of steps before 0 read as 0; column LT stays 0 for good
  {
    float4 *r4 = reinterpret_cast<float4 *>(ring);
    for (int i = lane; i < RR * RW / 4; i += LN) r4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  pass_sync<CL>();  // every CTA's ring is clear before any lane of the cluster reads one

  const int e_end = off[lg + 1];
  int e_nx = off[lg];  // index of the next row's entry
  int4 nxa = make_int4(0, 0, 0, 0), nxb = make_int4(0, 0, 0, 0);  // the next row's entry
  int ev = INT_MAX;  // the next row's switch step (its cursor event is kPackedPre steps earlier)
  if (e_nx < e_end) {
    nxa = ent[2 * e_nx];
    nxb = ent[2 * e_nx + 1];
    ev = nxa.x & 0xffff;
  }

  // position in the packed array of this pass's step s; the 16-byte block of
  // this lane holding steps 4g..4g+3 (backward: positions T-1-4g .. T-4-4g,
  // the block's elements in reverse order)
  auto ppos = [&](int s) { return FWD ? s : T - 1 - s; };
  auto block = [&](int g) {
    return reinterpret_cast<float4 *>(pw) + (size_t)(FWD ? g : (T >> 2) - 1 - g) * LT + lg;
  };

  // prefetch cursor: the far producers of the row this lane works on
  // kPackedPre steps ahead (word offsets into pw of their next values)
  int pgm = 0, pf_end = -1, o0 = 0, o1 = 0, o2 = 0;
  // the cursor moves to the next row at step tau2 = its switch step: its far
  // producers, and the copies of its coefficients and of the entry after it
  auto cursor = [&](int tau2) {
    pgm = (nxa.x >> 20) & 7;
    const int lo = (nxa.x & 0xffff) + ((nxa.x >> 16) & 15);
    pf_end = lo + (nxa.y & 1023) - 1;
    auto pos0 = [&](int code) {  // the value read at step tau2
      return packed_index32(ppos(tau2 - ((code >> 10) & 0xfffff) + 1), code & 1023, LT);
    };
    if (pgm) {
      o0 = pos0(nxb.y);
      o1 = pos0(nxb.z);
      o2 = pos0(nxb.w);
    }
    const float4 *src = reinterpret_cast<const float4 *>(tab + (size_t)(((unsigned)nxa.w >> 15) & 0x7fffu) * SF2);
    float4 *dst = reinterpret_cast<float4 *>(my_stage);
#pragma unroll
    for (int i = 0; i < SF2 / 2; ++i) cpa16(dst + i, src + i);
    if (e_nx + 1 < e_end) {
      cpa16(&sent[2 * lane], &ent[2 * (e_nx + 1)]);
      cpa16(&sent[2 * lane + 1], &ent[2 * (e_nx + 1) + 1]);
    }
  };
  // the next value of a far producer (position offset o, one step on)
  auto next_pos = [&](int &o) {
    if (FWD) o += (o & 3) == 3 ? 4 * LT - 3 : 1;
    else o -= (o & 3) == 0 ? 4 * LT - 3 : 1;
  };
  auto prefetch = [&](int tau2) {  // one commit group per step
    if (pgm && tau2 <= pf_end) {
      float *d = reinterpret_cast<float *>(q + (tau2 & (QS - 1)) * LN + lane);
      if (pgm & 1) cpa<4>(d + 1, pw + o0);
      if (pgm & 2) cpa<4>(d + 2, pw + o1);
      if (pgm & 4) cpa<4>(d + 3, pw + o2);
      next_pos(o0);
      next_pos(o1);
      next_pos(o2);
    }
    cpa_commit();
  };
#pragma unroll 1
  for (int s = 0; s < PD; ++s) {
    if (s == ev) cursor(s);
    prefetch(s);
  }

  // current row
  int lo = 0, cn = 0, c_y = 0, c_z = 0;
  int gm = 0;                       // bit j: producer j comes through the queue
  int B0 = LT, B1 = LT, B2 = LT;    // ring word of each producer's read at the block's first step
  // CL > 1: the other CTA's ring in the cluster window (every result is
  // stored there too)
  const unsigned peer = CL > 1 ? cluster_addr(ring, rank ^ 1u) : 0u;
  float cv0 = 0.f, cv1 = 0.f, cv2 = 0.f;  // each producer's value of the last step
  float v1 = 0.f;                         // this lane's value of the last step
  float2 t2 = make_float2(0.f, 0.f);
  const float2 dt2 = FWD ? make_float2(2.f * hh, 2.f * hh) : make_float2(-2.f * hh, -2.f * hh);
  const float2 one2 = make_float2(1.f, 1.f);
  float2 c[4][DX + 1];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int k = 0; k <= DX; ++k) c[p][k] = make_float2(0.f, 0.f);

  auto switch_row = [&]() {  // on the next row's switch step
    lo = (nxa.x & 0xffff) + ((nxa.x >> 16) & 15);
    cn = nxa.y & 1023;
    c_y = (nxa.y >> 10) & 1023;
    c_z = nxa.y >> 20;
    B0 = nxa.z & 0x7fff;
    B1 = (nxa.z >> 15) & 0x7fff;
    B2 = nxa.w & 0x7fff;
    gm = (nxa.x >> 20) & 7;
    const float tt = __int_as_float(nxb.x);
    t2 = make_float2(tt, tt);
    const float4 *sv = reinterpret_cast<const float4 *>(my_stage);
#pragma unroll
    for (int k = 0; k <= DX; ++k) {
      const float4 a = sv[2 * k], b = sv[2 * k + 1];
      c[0][k] = make_float2(a.x, a.y);
      c[1][k] = make_float2(a.z, a.w);
      c[2][k] = make_float2(b.x, b.y);
      c[3][k] = make_float2(b.z, b.w);
    }
    ++e_nx;
    ev = INT_MAX;
    if (e_nx < e_end) {
      nxa = sent[2 * lane];
      nxb = sent[2 * lane + 1];
      ev = nxa.x & 0xffff;
    }
  };

  // one step (J = tau & (kPackedBlock - 1), a constant after unrolling): the
  // events, the far prefetch, the point; input r (forward) or the forward
  // result (backward); returns this lane's result (0 without a point)
  auto step = [&](int tau, int J, bool mir, int wb, float in) -> float {
    cpa_wait<PD - 1>();  // the far values of step tau are in
    if ((J & (Q - 1)) == Q - 1 && tau == ev) switch_row();
    if (((J + PD) & (Q - 1)) == Q - 1 && tau + PD == ev) cursor(tau + PD);
    prefetch(tau + PD);
    // each producer's second value of this step
    float r0 = ring[B0 + J * RW], r1 = ring[B1 + J * RW], r2 = ring[B2 + J * RW];
    if (gm) {
      const float4 qv = q[J * LN + lane];
      if (gm & 1) r0 = qv.y;
      if (gm & 2) r1 = qv.z;
      if (gm & 4) r2 = qv.w;
    }
    const float a0 = cv0, a1 = cv1, a2 = cv2;  // first values: last step's second values
    cv0 = r0;
    cv1 = r1;
    cv2 = r2;
    // the eight row polynomials at the point's row coordinate
    float L[8];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float2 v = c[p][DX];
#pragma unroll
      for (int k = DX - 1; k >= 0; --k) v = ffma2(v, t2, c[p][k]);
      L[2 * p] = v.x;
      L[2 * p + 1] = v.y;
    }
    const bool active = (unsigned)(tau - lo) < (unsigned)cn;
    float acc;
    if (FWD) {
      if constexpr (V1) {  // the stored exact L^p_d at a cell-boundary point
        const float *bndv = reinterpret_cast<const float *>(t.bnd);
        const int x = tau - lo + 1;
        if (active && bndv && on_cell_boundary(N, x, c_y, c_z)) {
          const float *rec = bndv + (size_t)bnd_record(t.bnd_off, N, x, c_y, c_z) * 8;
#pragma unroll
          for (int d = 0; d < 7; ++d) L[d] = rec[d];
        }
      }
      // producers (x, y-1, z) / (x+1, y-1, z); (x, y, z-1) / (x+1, y, z-1);
      // (x-1, y+1, z-1) / (x, y+1, z-1); the row's own (x-1, y, z); the
      // values already held come first, this step's reads last
      acc = in;
      acc = fmaf(-L[1], a0, acc);
      acc = fmaf(-L[5], a1, acc);
      acc = fmaf(-L[3], a2, acc);
      acc = fmaf(-L[0], v1, acc);
      acc = fmaf(-L[2], r0, acc);
      acc = fmaf(-L[6], r1, acc);
      acc = fmaf(-L[4], r2, acc);
    } else {
      if constexpr (V1) {  // stored exact 1/D^p at p, L^{p-d}_d where p - d is a cell-boundary point
        const float *bndv = reinterpret_cast<const float *>(t.bnd);
        const int x = cn + lo - tau;
        if (active && bndv) {
          if (on_cell_boundary(N, x, c_y, c_z)) L[0] = bndv[(size_t)bnd_record(t.bnd_off, N, x, c_y, c_z) * 8 + 7];
#pragma unroll
          for (int d = 0; d < kNumLower; ++d) {
            const int qx = x - dir_dx(d), qy = c_y - dir_dy(d), qz = c_z - dir_dz(d);
            if (in_interior(N, qx, qy, qz) && on_cell_boundary(N, qx, qy, qz))
              L[1 + d] = bndv[(size_t)bnd_record(t.bnd_off, N, qx, qy, qz) * 8 + d];
          }
        }
      }
      // p - s = (x, y+1, z) / p - se = (x-1, y+1, z); p - bc = (x, y, z+1) /
      // p - be = (x-1, y, z+1); p - bnw = (x+1, y-1, z+1) / p - bn = (x, y-1,
      // z+1); the row's own p - w = (x+1, y, z)
      acc = L[0] * in;
      acc = fmaf(-L[2], a0, acc);
      acc = fmaf(-L[6], a1, acc);
      acc = fmaf(-L[4], a2, acc);
      acc = fmaf(-L[1], v1, acc);
      acc = fmaf(-L[3], r0, acc);
      acc = fmaf(-L[7], r1, acc);
      acc = fmaf(-L[5], r2, acc);
    }
    t2 = ffma2(t2, one2, dt2);  // the next point's row coordinate (exact)
    const float out = active ? acc : 0.f;
    v1 = out;
    ring[wb + J * RW] = out;
    if (mir) ring[(RG + J) * RW + lg] = out;
    if constexpr (CL > 1) {  // the same words of the other CTA's ring (visible there after the barrier)
      st_cluster(peer + 4u * (unsigned)(wb + J * RW), out);
      if (mir) st_cluster(peer + 4u * (unsigned)((RG + J) * RW + lg), out);
    }
    if ((J & (Q - 1)) == Q - 1) pass_sync<CL>();  // every Q steps (producers are at least Q + 1 steps ahead)
    return out;
  };

  const int G = T / kPackedBlock, G4 = T >> 2;
  float4 cur = *block(0);  // inputs of steps 0..3 (the residual launch ended before this kernel)
#pragma unroll 1
  for (int g = 0; g < G; ++g) {
    const int tau0 = g * kPackedBlock;
    const bool mir = (g & (RG / kPackedBlock - 1)) == 0;  // ring rows 0..7: also write their mirror
    const int wb = (tau0 & (RG - 1)) * RW + lg;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g4 = 2 * g + h;
      const float4 nxt = g4 + 1 < G4 ? *block(g4 + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
      float4 res;
      if (FWD) {
        res.x = step(tau0 + 4 * h, 4 * h, mir, wb, cur.x);
        res.y = step(tau0 + 4 * h + 1, 4 * h + 1, mir, wb, cur.y);
        res.z = step(tau0 + 4 * h + 2, 4 * h + 2, mir, wb, cur.z);
        res.w = step(tau0 + 4 * h + 3, 4 * h + 3, mir, wb, cur.w);
      } else {  // positions descend: the block's last element is this pass's first step
        res.w = step(tau0 + 4 * h, 4 * h, mir, wb, cur.w);
        res.z = step(tau0 + 4 * h + 1, 4 * h + 1, mir, wb, cur.z);
        res.y = step(tau0 + 4 * h + 2, 4 * h + 2, mir, wb, cur.y);
        res.x = step(tau0 + 4 * h + 3, 4 * h + 3, mir, wb, cur.x);
      }
      // the results over their inputs (a step without a point writes 0)
      *block(g4) = res;
      cur = nxt;
    }
    // the producers' ring words at the next block's first step
    B0 += kPackedBlock * RW;
    B1 += kPackedBlock * RW;
    B2 += kPackedBlock * RW;
    if (B0 >= RG * RW) B0 -= RG * RW;
    if (B1 >= RG * RW) B1 -= RG * RW;
    if (B2 >= RG * RW) B2 -= RG * RW;
  }
  cpa_wait<0>();
  pass_sync<CL>();  // no CTA clears its ring for the next pass while another still reads it
}

// one cluster of CL CTAs per tet (CL consecutive blocks)
template <int DX, bool V1, int Q, int CL>
__global__ void __launch_bounds__(cta_lanes(CL), 1) packed_kernel(const DevTet *__restrict__ tets,
                                                                 const int *__restrict__ order) {
  extern __shared__ __align__(16) unsigned char smem[];
  // a packed launch that follows this one as its programmatic dependent (a
  // batch's next group) may be dispatched as soon as every CTA of this one
  // has started: this launch's CTAs take their SMs first
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int b = (int)blockIdx.x / CL;
  const int ti = order ? order[b] : b;
  const DevTet &t = tets[ti];
  packed_pass<true, DX, V1, Q, CL>(t, smem);
  packed_pass<false, DX, V1, Q, CL>(t, smem);
}

template <int DX, bool V1, int Q, int CL>
cudaError_t launch_one(const PackedLaunch &L, size_t smem, cudaStream_t st) {
  auto k = packed_kernel<DX, V1, Q, CL>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (CL == 1 && !L.after_packed) {
    k<<<L.ntets, cta_lanes(CL), smem, st>>>(L.tets, L.order);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.ntets * CL);
  cfg.blockDim = dim3(cta_lanes(CL));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (CL > 1) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = CL;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  if (L.after_packed) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  e = cudaLaunchKernelEx(&cfg, k, L.tets, L.order);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int DX>
cudaError_t launch_dx(const PackedLaunch &L, size_t smem, cudaStream_t st) {
  // the schedules: quantum 1 (up to level 6) and 2 (level 7) on one CTA,
  // quantum 4 on a cluster of two (level 8)
  switch (L.q * 4 + L.cl * 2 + (L.v1 ? 1 : 0) - 2) {
    case 4: return launch_one<DX, false, 1, 1>(L, smem, st);
    case 5: return launch_one<DX, true, 1, 1>(L, smem, st);
    case 8: return launch_one<DX, false, 2, 1>(L, smem, st);
    case 9: return launch_one<DX, true, 2, 1>(L, smem, st);
    case 18: return launch_one<DX, false, 4, 2>(L, smem, st);
    case 19: return launch_one<DX, true, 4, 2>(L, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

// Between the lexicographic grid and the packed array, over the residual
// chunk list (the residual launch's blocks): a warp per kResidualCPW
// consecutive 32-point chunks, the grid side coalesced.
template <typename TX>
__global__ void __launch_bounds__(256) packed_io_kernel(const DevTet *__restrict__ tets, const int2 *__restrict__ bmap,
                                                        int mode, TX *const *__restrict__ xs, TX *x1) {
  const int2 bm = bmap ? bmap[blockIdx.x] : make_int2(0, (int)blockIdx.x);
  const DevTet &t = tets[bm.x];
  float *pwv = t.pk.pw;
  if (!pwv) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = (bm.y * 8 + warp) * kResidualCPW;
  const int N = t.N, nch = t.nchunks;
  const int *chunks = t.chunks, *row_map = t.pk.row_map;
  TX *x = xs ? xs[bm.x] : x1;
  // every chunk's addresses and loads first (the kernel is bound by load latency)
  constexpr int C = kResidualCPW;
  int gi[C], slot[C];
  bool ok[C];
#pragma unroll
  for (int k = 0; k < C; ++k) {
    int xx = 0, y = 1, z = 1;
    ok[k] = false;
    if (c0 + k < nch) ok[k] = chunk_point(N, chunks[c0 + k], lane, xx, y, z);  // warp-uniform test
    if (ok[k]) {
      const int m = row_map[row_id32(N, y, z)];
      slot[k] = packed_index32((m & 0xfffff) + xx - 1, m >> 20, t.pk.lanes);
      gi[k] = row_start32(N, y, z) + xx;
    }
  }
  if (mode == 0) {
    float w[C];
    TX xo[C];
#pragma unroll
    for (int k = 0; k < C; ++k)
      if (ok[k]) {
        w[k] = pwv[slot[k]];
        xo[k] = x[gi[k]];
      }
#pragma unroll
    for (int k = 0; k < C; ++k)
      if (ok[k]) x[gi[k]] = xo[k] + (TX)w[k];
  } else {
    TX xi[C];
#pragma unroll
    for (int k = 0; k < C; ++k)
      if (ok[k]) xi[k] = x[gi[k]];
#pragma unroll
    for (int k = 0; k < C; ++k)
      if (ok[k]) pwv[slot[k]] = (float)xi[k];
  }
}

}  // namespace

size_t packed_smem_bytes(int reg, int cl) {
  const size_t LN = cta_lanes(cl);
  return (size_t)RR * ring_row(cl) * 4 + QS * LN * 16 + LN * 32 + LN * 4 * (reg + 1) * 8;
}

cudaError_t launch_packed(const PackedLaunch &L, cudaStream_t st) {
  if (L.ntets <= 0) return cudaSuccess;
  const size_t smem = packed_smem_bytes(L.reg, L.cl);
  switch (L.reg) {  // the packed row tables are padded to degree 3 or 6
    case 3: return launch_dx<3>(L, smem, st);
    case 6: return launch_dx<6>(L, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_packed_io(int mode, bool f64, const DevTet *tets, const int2 *bmap, int total_blocks,
                             void *const *xs, void *x1, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  if (f64)
    packed_io_kernel<double><<<total_blocks, 256, 0, st>>>(tets, bmap, mode, reinterpret_cast<double *const *>(xs),
                                                           reinterpret_cast<double *>(x1));
  else
    packed_io_kernel<float><<<total_blocks, 256, 0, st>>>(tets, bmap, mode, reinterpret_cast<float *const *>(xs),
                                                          reinterpret_cast<float *>(x1));
  return cudaGetLastError();
}

}  // namespace ilu
