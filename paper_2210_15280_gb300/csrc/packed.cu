// packed.cu -- packed substitution kernels of the FP32 sweeps (Alg. 2 of
// arXiv 2210.15280 with the V2 boundary rule; V1 as an option).
//
// One CTA of kPackedLanes threads per macro-tetrahedron runs the forward
// substitution
//     w^p = r^p - sum_{d in D_l, p+d interior} L~^p_d w^{p+d}
// and then the backward substitution
//     w^p <- D~^-1(p) w^p - sum_{d in D_l, p-d interior} L~^{p-d}_d w^{p-d},
// walking the steps of the tet's host-computed row schedule (packed.h): at
// step tau every lane computes one point of the row it owns (or idles), then
// the CTA meets at a block barrier.  No CTA waits on another.  Everything the
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
//   queue      the input of the next kPackedPre steps, plus the values of
//              producer rows that ran too far ahead for the ring, read back
//              from the packed array -- filled by cp.async;
//   stage      the next row's coefficients and the schedule entry after it,
//              filled by cp.async while the current row runs.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"
#include "packed.h"

namespace ilu {
namespace {

constexpr int LN = kPackedLanes, RG = kPackedRing, QS = kPackedQueue, PD = kPackedPre;
static_assert((RG & (RG - 1)) == 0 && (QS & (QS - 1)) == 0, "ring and queue sizes are powers of two");
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

// One substitution of one tet on one CTA.
//
// Lane state: the current row (first step, points, the centred-coordinate
// offset N - y - z, producer codes), and per producer the ring index of the
// value it reads next and the value it read last (a consumer's first value
// at a step is its second value of the step before, so one ring read or
// queue entry per producer and step suffices); the next row's schedule entry
// (staged).  A lane switches to its next row on the idle step before the
// row's first point; the row's coefficients are read from the stage at the
// first point, and the stage is refilled for the row after at the end of
// that step.  Steps run in blocks of four: at the start of block g each lane
// loads its inputs of block g + 1 (one 16-byte load), and at the end of
// block g it stores the block's four results over their inputs.
template <bool FWD, int DX, bool V1>
__device__ __forceinline__ void packed_pass(const DevTet &t, unsigned char *smem) {
  constexpr int SF2 = 4 * (DX + 1);  // float2 of a staged row: coefficient k of the four function pairs
  float *ring = reinterpret_cast<float *>(smem);                 // [RG][LN]
  float4 *q = reinterpret_cast<float4 *>(ring + RG * LN);        // [QS][LN] far producer values (.y .z .w)
  int4 *sent = reinterpret_cast<int4 *>(q + QS * LN);            // [LN][2]
  float2 *stage = reinterpret_cast<float2 *>(sent + 2 * LN);     // [LN][SF2]
  const int lane = threadIdx.x;
  const int N = t.N;
  const int4 *ent = FWD ? t.pk.ent_f : t.pk.ent_b;  // entry e at ent[2e], ent[2e + 1]
  const int *off = t.pk.off;
  const int T = t.pk.nsteps;  // a multiple of 4
  const float2 *tab = reinterpret_cast<const float2 *>(FWD ? t.pkF : t.pkB);
  float *pw = t.pk.pw;  // packed array; backward step tau works on forward step T - 1 - tau
  const float hh = (float)(0.5 * t.h);
  float2 *my_stage = stage + lane * SF2;

  const int e_end = off[lane + 1];
  int e_cur = off[lane] - 1;
  bool has_nxt = e_cur + 1 < e_end, stage_pending = false;
  int4 na = make_int4(0, 0, 0, 0), nb = make_int4(0, 0, 0, 0);  // the next row's entry
  // current row: none yet (its step range is empty)
  int c_start = -8, c_n = 0, c_K = 0, c_p0 = 0, c_p1 = 0, c_p2 = 0, c_far = 0;
  int c_y = 0, c_z = 0;  // read by boundary variant V1 only
  int s0 = lane, s1 = lane, s2 = lane;          // ring index of each producer's next value
  float cv0 = 0.f, cv1 = 0.f, cv2 = 0.f;        // each producer's value of the last step
  float v1 = 0.f;                               // this row's previous value
  float2 c[4][DX + 1];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int k = 0; k <= DX; ++k) c[p][k] = make_float2(0.f, 0.f);

  auto stage_rows = [&](int rid, int e_after) {  // coefficients of row rid, entry e_after
    const float4 *src = reinterpret_cast<const float4 *>(tab + (size_t)rid * SF2);
    float4 *dst = reinterpret_cast<float4 *>(my_stage);
#pragma unroll
    for (int i = 0; i < SF2 / 2; ++i) cpa16(dst + i, src + i);
    if (e_after < e_end) {
      cpa16(&sent[2 * lane], &ent[2 * e_after]);
      cpa16(&sent[2 * lane + 1], &ent[2 * e_after + 1]);
    }
  };
  if (has_nxt) {
    na = ent[2 * (e_cur + 1)];
    nb = ent[2 * (e_cur + 1) + 1];
    stage_rows(na.w, e_cur + 2);
  }
  cpa_commit();

  // Position in the packed array of this pass's step s, and the 16-byte
  // block of this lane holding steps 4g..4g+3 (backward: positions
  // T-1-4g .. T-4-4g, the block's elements in reverse order).
  auto ppos = [&](int s) { return FWD ? s : T - 1 - s; };
  auto block = [&](int g) {
    return reinterpret_cast<float4 *>(pw) + (size_t)(FWD ? g : (T >> 2) - 1 - g) * LN + lane;
  };
  // far producer values of the point this lane works on at step tau2; one
  // commit group per step (a producer's second value of step tau2 was written
  // at tau2 - k0 + 1 >= tau2 - kPackedPre - ... well before this copy)
  auto prefetch = [&](int tau2) {
    const bool uc = tau2 <= c_start + c_n - 1;
    const bool un = !uc && has_nxt && tau2 >= na.x - 1;
    if ((uc && c_far) || (un && nb.w)) {
      const int p0 = uc ? c_p0 : nb.x, p1 = uc ? c_p1 : nb.y, p2 = uc ? c_p2 : nb.z;
      float *d = reinterpret_cast<float *>(q + (tau2 & (QS - 1)) * LN + lane);
      if (pmode(p0) == kProdGlobal)
        cpa<4>(d + 1, pw + packed_index(ppos(tau2 - ((p0 >> 9) & 0x1fffff) + 1), p0 & 511));
      if (pmode(p1) == kProdGlobal)
        cpa<4>(d + 2, pw + packed_index(ppos(tau2 - ((p1 >> 9) & 0x1fffff) + 1), p1 & 511));
      if (pmode(p2) == kProdGlobal)
        cpa<4>(d + 3, pw + packed_index(ppos(tau2 - ((p2 >> 9) & 0x1fffff) + 1), p2 & 511));
    }
    cpa_commit();
  };
#pragma unroll 1
  for (int s = 0; s < PD; ++s) prefetch(s);

  // ring index of a producer's value at step tau + 1 - k0 (its second value at tau)
  auto ring_start = [&](int code, int tau) {
    return pmode(code) == kProdRing ? ((tau - ((code >> 9) & 31) + 1) & (RG - 1)) * LN + (code & 511) : lane;
  };

  // one step: the switch, the far prefetch, the point; input r (forward) or
  // the forward result (backward); returns this lane's result (0 if idle)
  auto step = [&](int tau, float in) -> float {
    cpa_wait<PD - 1>();  // the far values of step tau are in
    if (has_nxt && tau == na.x - 1) {  // switch to the next row (its idle step)
      ++e_cur;
      c_start = na.x;
      c_n = na.y & 1023;
      c_y = (na.y >> 10) & 1023;
      c_z = na.y >> 20;
      c_K = N - c_y - c_z;
      c_p0 = nb.x;
      c_p1 = nb.y;
      c_p2 = nb.z;
      c_far = nb.w;
      s0 = ring_start(c_p0, tau);
      s1 = ring_start(c_p1, tau);
      s2 = ring_start(c_p2, tau);
      has_nxt = e_cur + 1 < e_end;
      if (has_nxt) {
        na = sent[2 * lane];
        nb = sent[2 * lane + 1];
      }
      stage_pending = true;
    }
    const bool first = stage_pending && tau == c_start;
    if (first) {  // the row's coefficients from the stage
      const float4 *sv = reinterpret_cast<const float4 *>(my_stage);
#pragma unroll
      for (int k = 0; k <= DX; ++k) {
        const float4 a = sv[2 * k], b = sv[2 * k + 1];
        c[0][k] = make_float2(a.x, a.y);
        c[1][k] = make_float2(a.z, a.w);
        c[2][k] = make_float2(b.x, b.y);
        c[3][k] = make_float2(b.z, b.w);
      }
    }
    prefetch(tau + PD);
    float out = 0.f;
    if (tau >= c_start - 1 && tau <= c_start + c_n - 1) {
      const float4 qv = q[(tau & (QS - 1)) * LN + lane];
      // each producer's second value of this step: ring, queue or none
      const float r0 = ring[s0], r1 = ring[s1], r2 = ring[s2];
      const float b0 = pmode(c_p0) == kProdRing ? r0 : (pmode(c_p0) == kProdGlobal ? qv.y : 0.f);
      const float b1 = pmode(c_p1) == kProdRing ? r1 : (pmode(c_p1) == kProdGlobal ? qv.z : 0.f);
      const float b2 = pmode(c_p2) == kProdRing ? r2 : (pmode(c_p2) == kProdGlobal ? qv.w : 0.f);
      const float a0 = cv0, a1 = cv1, a2 = cv2;  // first values: last step's second values
      cv0 = b0;
      cv1 = b1;
      cv2 = b2;
      s0 = s0 + LN < RG * LN ? s0 + LN : s0 + LN - RG * LN;
      s1 = s1 + LN < RG * LN ? s1 + LN : s1 + LN - RG * LN;
      s2 = s2 + LN < RG * LN ? s2 + LN : s2 + LN - RG * LN;
      if (tau >= c_start) {
        const int u = tau - c_start + 1;
        const int x = FWD ? u : c_n + 1 - u;
        // the eight row polynomials at the centred row coordinate
        float L[8];
        {
          const float tt = (float)(2 * x - c_K) * hh;
          const float2 t2 = make_float2(tt, tt);
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            float2 v = c[p][DX];
#pragma unroll
            for (int k = DX - 1; k >= 0; --k) v = ffma2(v, t2, c[p][k]);
            L[2 * p] = v.x;
            L[2 * p + 1] = v.y;
          }
        }
        const float zero = 0.f;
        float acc;
        if (FWD) {
          if constexpr (V1) {  // the stored exact L^p_d at a cell-boundary point
            const float *bndv = reinterpret_cast<const float *>(t.bnd);
            if (bndv && on_cell_boundary(N, x, c_y, c_z)) {
              const float *rec = bndv + (size_t)bnd_record(t.bnd_off, N, x, c_y, c_z) * 8;
#pragma unroll
              for (int d = 0; d < 7; ++d) L[d] = rec[d];
            }
          }
          const bool x2 = x >= 2;
          const float ws = a0, wse = b0;                  // (x, y-1, z), (x+1, y-1, z): none if y = 1
          const float wbc = a1, wbe = b1;                 // (x, y, z-1), (x+1, y, z-1): none if z = 1
          const float wbnw = x2 ? a2 : zero, wbn = b2;    // (x-1, y+1, z-1), (x, y+1, z-1)
          const float ww = x2 ? v1 : zero;                // (x-1, y, z)
          acc = in;
          acc = fmaf(-L[1], ws, acc);
          acc = fmaf(-L[2], wse, acc);
          acc = fmaf(-L[3], wbnw, acc);
          acc = fmaf(-L[4], wbn, acc);
          acc = fmaf(-L[5], wbc, acc);
          acc = fmaf(-L[6], wbe, acc);
          acc = fmaf(-L[0], ww, acc);
        } else {
          if constexpr (V1) {  // stored exact 1/D^p at p, L^{p-d}_d where p - d is a cell-boundary point
            const float *bndv = reinterpret_cast<const float *>(t.bnd);
            if (bndv) {
              if (on_cell_boundary(N, x, c_y, c_z))
                L[0] = bndv[(size_t)bnd_record(t.bnd_off, N, x, c_y, c_z) * 8 + 7];
#pragma unroll
              for (int d = 0; d < kNumLower; ++d) {
                const int qx = x - dir_dx(d), qy = c_y - dir_dy(d), qz = c_z - dir_dz(d);
                if (in_interior(N, qx, qy, qz) && on_cell_boundary(N, qx, qy, qz))
                  L[1 + d] = bndv[(size_t)bnd_record(t.bnd_off, N, qx, qy, qz) * 8 + d];
              }
            }
          }
          const bool inner = u >= 2, x2 = x >= 2;         // x + y + z <= N - 2; x >= 2
          const float wn = inner ? a0 : zero;             // p - s   = (x, y+1, z)
          const float wnw = x2 ? b0 : zero;               // p - se  = (x-1, y+1, z)
          const float wtc = inner ? a1 : zero;            // p - bc  = (x, y, z+1)
          const float wtw = x2 ? b1 : zero;               // p - be  = (x-1, y, z+1)
          const float wtse = inner ? a2 : zero;           // p - bnw = (x+1, y-1, z+1): none if y = 1
          const float wts = b2;                           // p - bn  = (x, y-1, z+1): none if y = 1
          const float we = inner ? v1 : zero;             // p - w   = (x+1, y, z)
          acc = L[0] * in;
          acc = fmaf(-L[2], wn, acc);
          acc = fmaf(-L[6], wtc, acc);
          acc = fmaf(-L[4], wtse, acc);
          acc = fmaf(-L[3], wnw, acc);
          acc = fmaf(-L[7], wtw, acc);
          acc = fmaf(-L[5], wts, acc);
          acc = fmaf(-L[1], we, acc);
        }
        ring[(tau & (RG - 1)) * LN + lane] = acc;
        v1 = acc;
        out = acc;
      }
    }
    if (first) {  // the stage is read (its values are in use): refill it for the row after
      if (has_nxt) stage_rows(na.w, e_cur + 2);
      stage_pending = false;
    }
    __syncthreads();
    return out;
  };

  const int G = T >> 2;
  float4 cur = *block(0);  // inputs of block 0 (the residual launch ended before this kernel)
#pragma unroll 1
  for (int g = 0; g < G; ++g) {
    const float4 nxt = g + 1 < G ? *block(g + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 res;
    if (FWD) {
      res.x = step(4 * g, cur.x);
      res.y = step(4 * g + 1, cur.y);
      res.z = step(4 * g + 2, cur.z);
      res.w = step(4 * g + 3, cur.w);
    } else {  // positions descend: the block's last element is this pass's first step
      res.w = step(4 * g, cur.w);
      res.z = step(4 * g + 1, cur.z);
      res.y = step(4 * g + 2, cur.y);
      res.x = step(4 * g + 3, cur.x);
    }
    // the block's results over its inputs; an idle step keeps its slot's value
    // (a slot without a point holds no value anyone reads)
    *block(g) = res;
    cur = nxt;
  }
  cpa_wait<0>();
  __syncthreads();
}

template <int DX, bool V1>
__global__ void __launch_bounds__(kPackedLanes, 1) packed_kernel(const DevTet *__restrict__ tets,
                                                                 const int *__restrict__ order) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ti = order ? order[blockIdx.x] : (int)blockIdx.x;
  const DevTet &t = tets[ti];
  packed_pass<true, DX, V1>(t, smem);
  packed_pass<false, DX, V1>(t, smem);
}

template <int DX>
cudaError_t launch_dx(const PackedLaunch &L, size_t smem, cudaStream_t st) {
  auto k = L.v1 ? packed_kernel<DX, true> : packed_kernel<DX, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<L.ntets, kPackedLanes, smem, st>>>(L.tets, L.order);
  return cudaGetLastError();
}

// Between the lexicographic grid and the packed array, over the residual
// chunk list (the residual launch's blocks): a warp per kResidualCPW
// consecutive 32-point row chunks, the grid side coalesced.
template <typename TX>
__global__ void __launch_bounds__(256) packed_io_kernel(const DevTet *__restrict__ tets, const int *__restrict__ bprefix,
                                                        int n, int mode, TX *const *__restrict__ xs, TX *x1) {
  int lo = 0;
  if (bprefix) {
    int hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (bprefix[mid] <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
  }
  const DevTet &t = tets[lo];
  if (!t.pk.pw) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = (((int)blockIdx.x - (bprefix ? bprefix[lo] : 0)) * 8 + warp) * kResidualCPW;
  const int N = t.N;
  TX *x = xs ? xs[lo] : x1;
#pragma unroll 1
  for (int k = 0; k < kResidualCPW && c0 + k < t.nchunks; ++k) {
    const int ch = t.chunks[c0 + k];
    const int y = (ch >> 10) & 1023, z = ch >> 20, xx = 1 + 32 * (ch & 1023) + lane;
    if (xx > N - 1 - y - z) continue;
    const int m = t.pk.row_map[row_id(N, y, z)];
    float *slot = t.pk.pw + packed_index((m & 0xfffff) + xx - 1, m >> 20);
    const int64_t gi = grid_index(N, xx, y, z);
    if (mode == 0) x[gi] = x[gi] + (TX)*slot;
    else *slot = (float)x[gi];
  }
}

}  // namespace

size_t packed_smem_bytes(int reg) {
  return (size_t)RG * LN * 4 + (size_t)QS * LN * 16 + (size_t)LN * 32 + (size_t)LN * 4 * (reg + 1) * 8;
}

cudaError_t launch_packed(const PackedLaunch &L, cudaStream_t st) {
  if (L.ntets <= 0) return cudaSuccess;
  const size_t smem = packed_smem_bytes(L.reg);
  switch (L.reg) {  // the packed row tables are padded to degree 3 or 6
    case 3: return launch_dx<3>(L, smem, st);
    case 6: return launch_dx<6>(L, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_packed_io(int mode, bool f64, const DevTet *tets, const int *bprefix, int ntets, int total_blocks,
                             void *const *xs, void *x1, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  if (f64)
    packed_io_kernel<double><<<total_blocks, 256, 0, st>>>(tets, bprefix, ntets, mode,
                                                           reinterpret_cast<double *const *>(xs),
                                                           reinterpret_cast<double *>(x1));
  else
    packed_io_kernel<float><<<total_blocks, 256, 0, st>>>(tets, bprefix, ntets, mode,
                                                          reinterpret_cast<float *const *>(xs),
                                                          reinterpret_cast<float *>(x1));
  return cudaGetLastError();
}

}  // namespace ilu
