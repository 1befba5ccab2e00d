// band.cu -- FP32 substitutions of Alg. 2 (arXiv 2210.15280) with one row per
// lane and no block-wide synchronisation.
//
// Layout.  The sweep keeps r/w in a band-major array: band (z,k) (grid.h) is
// a [step][32 lanes] block, entry (s, j) holding the point x = s - 2j of row
// band_Y(z,k) + j.  Every step of a band is one coalesced 128-byte line.
// band_residual_kernel writes r there (transposing through shared memory),
// band_update_kernel adds the result to x the same way.
//
// Substitutions.  A CTA is a stack of Z consecutive layers of one band, one
// warp per layer; a warp walks the steps of its band (forward: increasing,
// backward: decreasing).  Dependencies (forward; the backward mirrors them):
//   same row, previous step                 register
//   row y-1 (lane j-1), steps s-1, s-2      shuffle; lane 0: band k-1, lane 31,
//                                           through its stream in global memory
//   layer z-1 (same band), steps s..s-2     the warp below: a shared-memory ring;
//                                           the bottom warp: the CTA below,
//                                           through a per-step stream in global
//   layer z-1, row y (lane 0)               band k-1 of layer z-1, its stream
// An edge stream holds 16-byte records: record s = the edge lane's values at
// steps s and s+1, which is the pair a neighbour needs at one step.
// Exchanged words carry a tag next to the value (one 8-byte store), so a
// reader checks the tag instead of waiting on a separate flag: no fences,
// and a producer that is ahead costs the reader nothing.  Global streams are
// written once per launch and tagged with the launch's epoch; ring slots are
// reused and tagged with the step.  The reader prefetches global words a few
// steps ahead with cp.async and falls back to polling only if a tag is not
// there yet.  CTAs take tickets in dependency order, so every wait is on a
// CTA that is resident or finished.  Every wait is bounded.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <utility>

#include "../../include/ilu.h"
#include "kernels.cuh"
#include "stencil.cuh"

namespace ilu {

namespace {

constexpr int kRing = 16;   // ring slots per warp (shared memory)
constexpr int kPre = 12;    // prefetch distance in steps
constexpr int kQ = 16;      // prefetch slots (> kPre)
// Tagged words from other CTAs are fetched only 2 steps ahead: a consumer
// runs just behind its producer, and a word fetched earlier than the hop
// latency would always be stale.

// ------------------------------------------------------------- primitives --

__device__ __forceinline__ unsigned long long ll_pack(float v, unsigned tag) {
  return (unsigned long long)__float_as_uint(v) | ((unsigned long long)tag << 32);
}
__device__ __forceinline__ float ll_val(unsigned long long w) { return __uint_as_float((unsigned)w); }
__device__ __forceinline__ unsigned ll_tag(unsigned long long w) { return (unsigned)(w >> 32); }

__device__ __forceinline__ void st_ll_global(unsigned long long *p, unsigned long long w) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ unsigned long long ld_ll_global(const unsigned long long *p) {
  unsigned long long w;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
  return w;
}
template <int BYTES>
__device__ __forceinline__ void cpa(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src),
               "n"(BYTES)
               : "memory");
}
// two tagged words in one store (each 8-byte half is a single-copy-atomic word)
__device__ __forceinline__ void st_ll2_global(unsigned long long *p, unsigned long long a, unsigned long long b) {
  asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
// predicated forms (no branch in the step loop)
__device__ __forceinline__ void cpa4_if(bool p, void *dst, const void *src) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q cp.async.ca.shared.global [%0], [%1], 4;\n\t}" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"((int)p)
               : "memory");
}
__device__ __forceinline__ void st_ll2_if(bool p, unsigned long long *a, unsigned long long u, unsigned long long v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t@q st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};\n\t}" ::"l"(a),
               "l"(u), "l"(v), "r"((int)p)
               : "memory");
}
__device__ __forceinline__ void st_f32_if(bool p, float *a, float v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.global.f32 [%0], %1;\n\t}" ::"l"(a), "f"(v), "r"((int)p)
               : "memory");
}
__device__ __forceinline__ unsigned long long ld_ll_if(bool p, const unsigned long long *a, unsigned long long dflt) {
  unsigned long long v = dflt;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q ld.relaxed.gpu.global.b64 %0, [%1];\n\t}"
               : "+l"(v) : "l"(a), "r"((int)p) : "memory");
  return v;
}
__device__ __forceinline__ ulonglong2 ld_ll2_if(bool p, const unsigned long long *a, ulonglong2 dflt) {
  unsigned long long x = dflt.x, y = dflt.y;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t@q ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];\n\t}"
               : "+l"(x), "+l"(y) : "l"(a), "r"((int)p) : "memory");
  return make_ulonglong2(x, y);
}
__device__ __forceinline__ unsigned long long ld_ring(const unsigned long long *a) {
  unsigned long long v;
  asm volatile("ld.volatile.shared.b64 %0, [%1];" : "=l"(v) : "r"((unsigned)__cvta_generic_to_shared(a)) : "memory");
  return v;
}
__device__ __forceinline__ void st_ring(unsigned long long *a, unsigned long long v) {
  asm volatile("st.volatile.shared.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(a)), "l"(v) : "memory");
}
__device__ __forceinline__ void st_hint_if(bool p, int *a, int v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.volatile.shared.s32 [%0], %1;\n\t}" ::"r"(
                   (unsigned)__cvta_generic_to_shared(a)),
               "r"(v), "r"((int)p)
               : "memory");
}
// a ring word of step s: the tag is the step (slots are reused); the hint
// said it is there, so a miss is rare and short
__device__ __forceinline__ float ring_value(const unsigned long long *a, unsigned s, const int *flag) {
  unsigned long long w = ld_ring(a);
  int spins = 0;
  while (ll_tag(w) != s) {
    if (*(volatile int *)flag || ++spins > (1 << 24)) return 0.f;
    w = ld_ring(a);
  }
  return ll_val(w);
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
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

// the eight row polynomials of one lane, degree DX, in registers (pair layout:
// coefficient k of functions 2p, 2p+1 at float2 index p*DXP + k)
template <int DX>
struct Row8 {
  float2 c[4][DX + 1];
  template <int DXP>
  __device__ __forceinline__ void load(const float *row) {
    const float2 *q = reinterpret_cast<const float2 *>(row);
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int k = 0; k <= DX; ++k) c[p][k] = q[p * DXP + k];
  }
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int k = 0; k <= DX; ++k) c[p][k] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void eval(float t, float (&out)[8]) const {
    const float2 t2 = make_float2(t, t);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float2 v = c[p][DX];
#pragma unroll
      for (int k = DX - 1; k >= 0; --k) v = fma2(v, t2, c[p][k]);
      out[2 * p] = v.x;
      out[2 * p + 1] = v.y;
    }
  }
};

// A wait that runs out records where (first one only), raises the CTA's
// abort flag in shared memory and returns; every warp leaves its step loop
// when it sees the flag.
__device__ __noinline__ void give_up(int *flag, LaunchStatus *st, int where, int level) {
  if (atomicCAS(&st->code, 0, (int)ILU_ETIMEOUT) == 0) {
    st->where = where;
    st->level = level;
  }
  atomicExch(flag, 1);
}

// value of a global stream word whose prefetched copy is stale: poll until
// the tag is there (bounded); 0 on give-up
__device__ __noinline__ float poll_global(const unsigned long long *p, unsigned tag, int *flag, LaunchStatus *st,
                                          long long max_spins, int where, int level) {
  long long spins = 0;
  for (;;) {
    const unsigned long long w = ld_ll_global(p);
    if (ll_tag(w) == tag) return ll_val(w);
    if (*(volatile int *)flag) return 0.f;
    if (++spins > max_spins) {
      give_up(flag, st, where, level);
      return 0.f;
    }
    if ((spins & 63) == 0 && *(volatile int *)&st->code) {  // another CTA gave up: so does this one
      atomicExch(flag, 1);
      return 0.f;
    }
    if (spins > 4) __nanosleep(spins < 64 ? 64 : 256);
  }
}
// one lane waits until a progress word reaches `need` (forward: >= need,
// backward: <= need), sleeping between reads; returns the last value seen.
// Progress words are hints that keep the other 31 lanes and the tag polls
// off the shared-memory pipe; the per-word tags still decide.
__device__ __noinline__ int wait_hint(const int *word, int need, bool ge, int *flag, LaunchStatus *st,
                                      long long max_spins, int where, int level) {
  long long spins = 0;
  for (;;) {
    const int v = *(const volatile int *)word;
    if (ge ? v >= need : v <= need) return v;
    if (*(volatile int *)flag) return v;
    if (++spins > max_spins) {
      give_up(flag, st, where, level);
      return v;
    }
    if ((spins & 63) == 0 && *(volatile int *)&st->code) {
      atomicExch(flag, 1);
      return v;
    }
    __nanosleep(spins < 8 ? 20 : 64);
  }
}
// back-pressure: wait until the consumer's progress word passes `need`
// (forward: >= need, backward: <= need); false on give-up
__device__ __noinline__ bool wait_progress(const int *word, int need, bool ge, int *flag, LaunchStatus *st,
                                           long long max_spins, int where, int level, int *seen) {
  long long spins = 0;
  for (;;) {
    const int v = *(const volatile int *)word;
    if (ge ? v >= need : v <= need) {
      *seen = v;
      return true;
    }
    if (*(volatile int *)flag) return false;
    if (++spins > max_spins) {
      give_up(flag, st, where, level);
      return false;
    }
    if ((spins & 63) == 0 && *(volatile int *)&st->code) {
      atomicExch(flag, 1);
      return false;
    }
    if (spins > 4) __nanosleep(32);
  }
}

// CTA c of a tet: group g = cta >> 16, band k = cta & 0xffff
__device__ __forceinline__ int owner_of(const BatchMap &bm, int ticket) {
  int lo = 0, hi = bm.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bm.prefix[mid] <= ticket) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------ forward --

template <int DXP, int REG, bool V1>
__global__ void __launch_bounds__(256, 2) fwd_band(const DevTet *__restrict__ tets, BatchMap bm,
                                                   LaunchStatus *status, long long max_spins) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int Z = blockDim.x >> 5;
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long *ring = reinterpret_cast<unsigned long long *>(smem);     // [Z][kRing][32] tagged values for the next warp
  float *rq = reinterpret_cast<float *>(ring + (size_t)Z * kRing * 32);         // [Z][kQ][32] prefetched inputs
  int *prog = reinterpret_cast<int *>(rq + (size_t)Z * kQ * 32);                // [Z] consumer progress
  int *done = prog + Z;                                                         // [Z] producer progress
  __shared__ int s_ticket, s_abort;
  if (threadIdx.x == 0) {
    s_ticket = atomicAdd(bm.ticket, 1);
    s_abort = 0;
  }
  for (int i = threadIdx.x; i < Z * kRing * 32; i += blockDim.x) ring[i] = ll_pack(0.f, 0x80000000u);
  if (threadIdx.x < Z) {
    prog[threadIdx.x] = INT_MIN;
    done[threadIdx.x] = INT_MIN;
  }
  __syncthreads();
  const int owner = owner_of(bm, s_ticket);
  const DevTet &t = tets[bm.order[owner]];
  const int cta = t.band.cta[s_ticket - bm.prefix[owner]];
  const int g = cta >> 16, k = cta & 0xffff;
  const int N = t.N;
  const int z = 1 + g * Z + wi;
    if (band_exists(N, z, k)) {
    const unsigned epoch = (unsigned)t.band.epoch[0] - 1u;  // forward: odd epochs
    const BandInfo bi = t.band.info[(size_t)(z - 1) * (band_kmax(N) + 1) + k];
    const int Y = band_Y(z, k), y = Y + lane;
    const bool row_ok = y >= 1 && y <= N - 2 - z;
    const int n = N - 1 - y - z;
    const int shi = band_shi(N, z, k);
    const int slo_self = band_slo(z, k);
    const int sbeg = z >= 2 ? band_slo(z - 1, k) : slo_self;  // the layer below starts earlier
    float *wb = reinterpret_cast<float *>(t.band.w) + bi.off;        // [step-1][32]
    unsigned long long *hs_out = t.band.streams + bi.hoff;           // lane 31 -> band k+1
    const bool top = wi == Z - 1 || !band_exists(N, z + 1, k);
    unsigned long long *vs_out = (top && bi.voff >= 0) ? t.band.streams + bi.voff : nullptr;  // [step][32]
    // inputs from outside the CTA
    const bool bottom = wi == 0 && z >= 2;
    const unsigned long long *vs_in = nullptr;
    if (bottom) {
      const BandInfo bb = t.band.info[(size_t)(z - 2) * (band_kmax(N) + 1) + k];
      vs_in = t.band.streams + bb.voff;
    }
    const bool need_s = row_ok && lane == 0 && y >= 2;    // s, se from band k-1 of this layer
    const bool need_b = row_ok && lane == 0 && z >= 2;    // bc, be from band k-1 of layer z-1
    const bool has_edge = __shfl_sync(0xffffffffu, need_s || need_b, 0);
    const unsigned long long *hs_left = nullptr, *hs_diag = nullptr;
    if (need_s) hs_left = t.band.streams + t.band.info[(size_t)(z - 1) * (band_kmax(N) + 1) + k - 1].hoff;
    if (need_b) hs_diag = t.band.streams + t.band.info[(size_t)(z - 2) * (band_kmax(N) + 1) + k - 1].hoff;
    Row8<(REG >= 0 ? REG : 0)> C;
    if (row_ok) C.template load<DXP>(reinterpret_cast<const float *>(t.tabF) + (size_t)row_id(N, y, z) * 8 * DXP);
    else C.zero();
    const float hh = (float)(0.5 * t.h);
    unsigned long long *my_ring = ring + (size_t)wi * kRing * 32;
    const unsigned long long *below_ring = wi > 0 ? ring + (size_t)(wi - 1) * kRing * 32 : nullptr;
    float *my_rq = rq + (size_t)wi * kQ * 32;

    auto prefetch = [&](int s) {
      if (s >= sbeg && s <= shi) cpa4_if(true, my_rq + (s & (kQ - 1)) * 32 + lane, wb + (size_t)(s - 1) * 32 + lane);
      cpa_commit();
    };
    for (int s = sbeg; s < sbeg + kPre; ++s) prefetch(s);
    // tagged words of step s+1, s+2 in flight (V: bottom warp; edges: lane 0)
    const ulonglong2 none2 = make_ulonglong2(0ull, 0ull);
    auto fetch_v = [&](int s) { return ld_ll_if(bottom && s <= shi, vs_in + (size_t)s * 32 + lane, 0ull); };
    auto fetch_l = [&](int s) { return ld_ll2_if(need_s && s <= shi, hs_left + 2 * (s + 62), none2); };
    auto fetch_d = [&](int s) { return ld_ll2_if(need_b && s <= shi, hs_diag + 2 * (s + 62), none2); };
    unsigned long long vq1 = fetch_v(sbeg), vq2 = fetch_v(sbeg + 1);
    ulonglong2 lq1 = fetch_l(sbeg), lq2 = fetch_l(sbeg + 1), dq1 = fetch_d(sbeg), dq2 = fetch_d(sbeg + 1);

    float v1 = 0.f, v2 = 0.f;            // this lane's values at steps s-1, s-2
    float b1 = 0.f, b2 = 0.f;            // layer below, this lane's column, steps s-1, s-2
    int cons_seen = INT_MIN;             // progress of the warp above (ring reuse)
    int below_seen = INT_MIN;            // progress of the warp below (ring fill)
    for (int s = sbeg; s <= shi; ++s) {
      prefetch(s + kPre);
      cpa_wait<kPre>();
      const int slot = s & (kQ - 1);
      const int x = s - 2 * lane;
      const bool act = row_ok && x >= 1 && x <= n;
      // layer below, this lane's column at step s (branches on warp-uniform conditions only)
      float b0 = 0.f;
      if (z >= 2) {
        unsigned long long w;
        if (wi > 0) {
          // the warp below published step s (release/acquire on its progress word)
          if (below_seen < s) {
            int v = 0;
            if (lane == 0) v = wait_hint(&done[wi - 1], s, true, &s_abort, status, max_spins, z, s);
            below_seen = __shfl_sync(0xffffffffu, v, 0);
            if (below_seen < s) break;  // gave up
          }
          b0 = ring_value(below_ring + (s & (kRing - 1)) * 32 + lane, (unsigned)s, &s_abort);
        } else {
          w = vq1;
          const bool ok = ll_tag(w) == epoch;
          if (!__all_sync(0xffffffffu, ok)) {
            if (!ok) w = ll_pack(poll_global(vs_in + (size_t)s * 32 + lane, epoch, &s_abort, status, max_spins, z, s), epoch);
            if (__shfl_sync(0xffffffffu, *(volatile int *)&s_abort, 0)) break;
          }
          b0 = ll_val(w);
        }
      }
      // neighbours in lane j-1; lane 0 takes them from band k-1 (edge words, all lanes load the broadcast)
      float ws = __shfl_up_sync(0xffffffffu, v2, 1);   // (x, y-1, z)
      float wse = __shfl_up_sync(0xffffffffu, v1, 1);  // (x+1, y-1, z)
      float wbc = __shfl_up_sync(0xffffffffu, b2, 1);  // (x, y, z-1)
      float wbe = __shfl_up_sync(0xffffffffu, b1, 1);  // (x+1, y, z-1)
      if (has_edge) {  // uniform: lane 0 of this warp needs band k-1
        unsigned long long e0 = lq1.x, e1 = lq1.y;
        unsigned long long e2 = dq1.x, e3 = dq1.y;
        const bool use_s = need_s && act, use_b = need_b && act;
        const bool ok = (!use_s || (ll_tag(e0) == epoch && ll_tag(e1) == epoch)) &&
                        (!use_b || (ll_tag(e2) == epoch && ll_tag(e3) == epoch));
        if (!__all_sync(0xffffffffu, ok)) {
          if (!ok) {
            if (use_s) {
              if (ll_tag(e0) != epoch) e0 = ll_pack(poll_global(hs_left + 2 * (s + 62), epoch, &s_abort, status, max_spins, z, s), epoch);
              if (ll_tag(e1) != epoch) e1 = ll_pack(poll_global(hs_left + 2 * (s + 62) + 1, epoch, &s_abort, status, max_spins, z, s), epoch);
            }
            if (use_b) {
              if (ll_tag(e2) != epoch) e2 = ll_pack(poll_global(hs_diag + 2 * (s + 62), epoch, &s_abort, status, max_spins, z, s), epoch);
              if (ll_tag(e3) != epoch) e3 = ll_pack(poll_global(hs_diag + 2 * (s + 62) + 1, epoch, &s_abort, status, max_spins, z, s), epoch);
            }
          }
          if (__shfl_sync(0xffffffffu, *(volatile int *)&s_abort, 0)) break;
        }
        if (lane == 0) {
          ws = ll_val(e0);
          wse = ll_val(e1);
          wbc = ll_val(e2);
          wbe = ll_val(e3);
        }
      }
      // w^p = r^p - sum_{d in D_l, p+d interior} L~^p_d w^{p+d}, evaluated on
      // every lane; terms of neighbours outside the interior are selected
      // away (V2), the previous step of this row goes last (shortest chain)
      float L[8];
      C.eval((float)(2 * x - (N - y - z)) * hh, L);
      if constexpr (V1) {  // boundary variant V1: the stored exact L^p_d at a cell-boundary point p
        const float *bndv = reinterpret_cast<const float *>(t.bnd);
        if (bndv && act && on_cell_boundary(N, x, y, z)) {
          const float *rec = bndv + (size_t)bnd_record(t.bnd_off, N, x, y, z) * 8;
#pragma unroll
          for (int d = 0; d < 7; ++d) L[d] = rec[d];
        }
      }
      const float zero = 0.f;
      ws = y >= 2 ? ws : zero;
      wse = y >= 2 ? wse : zero;
      const bool zb2 = z >= 2;
      const float wbnw = (zb2 && x >= 2) ? b1 : zero;
      const float wbn = zb2 ? b0 : zero;
      wbc = zb2 ? wbc : zero;
      wbe = zb2 ? wbe : zero;
      const float ww = x >= 2 ? v1 : zero;
      float acc = my_rq[slot * 32 + lane];
      acc = fmaf(-L[1], ws, acc);
      acc = fmaf(-L[2], wse, acc);
      acc = fmaf(-L[3], wbnw, acc);
      acc = fmaf(-L[4], wbn, acc);
      acc = fmaf(-L[5], wbc, acc);
      acc = fmaf(-L[6], wbe, acc);
      acc = fmaf(-L[0], ww, acc);
      const float val = act ? acc : zero;
      st_f32_if(act, wb + (size_t)(s - 1) * 32 + lane, val);
      // publish: the warp above (ring), the band above in the next CTA, band k+1
      if (top) {
        if (vs_out) st_ll_global(vs_out + (size_t)s * 32 + lane, ll_pack(val, epoch));
      } else {
        // the slot last held step s - kRing; the warp above reads steps from
        // band_slo(z, k) on, so an earlier one was never read
        if (s - kRing >= slo_self && cons_seen < s - kRing) {
          int seen = cons_seen;
          if (lane == 0) wait_progress(&prog[wi + 1], s - kRing, true, &s_abort, status, max_spins, z, s, &seen);
          cons_seen = __shfl_sync(0xffffffffu, seen, 0);
          if (cons_seen < s - kRing) break;  // gave up
        }
        st_ring(my_ring + (s & (kRing - 1)) * 32 + lane, ll_pack(val, (unsigned)s));
        st_hint_if(lane == 0, &done[wi], s);
      }
      st_ll2_if(lane == 31, hs_out + 2 * (s - 1), ll_pack(v1, epoch), ll_pack(val, epoch));  // record s-1
      st_hint_if(lane == 0 && wi > 0, &prog[wi], s);
      v2 = v1;
      v1 = val;
      b2 = b1;
      b1 = b0;
      vq1 = vq2;
      vq2 = fetch_v(s + 2);
      lq1 = lq2;
      lq2 = fetch_l(s + 2);
      dq1 = dq2;
      dq2 = fetch_d(s + 2);
    }
    st_hint_if(lane == 0 && wi > 0, &prog[wi], INT_MAX);  // no more ring reads
    cpa_wait<0>();
  }
}

// ----------------------------------------------------------- backward --

// w^p <- D~^{-1}(p) w^p - sum_{d in D_l, p-d interior} L~^{p-d}_d w^{p-d},
// in decreasing step order; the result stays in the band array (x is
// updated by band_update_kernel).
template <int DXP, int REG, bool V1>
__global__ void __launch_bounds__(256, 2) bwd_band(const DevTet *__restrict__ tets, BatchMap bm,
                                                   LaunchStatus *status, long long max_spins) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int Z = blockDim.x >> 5;
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long *ring = reinterpret_cast<unsigned long long *>(smem);     // [Z][kRing][32] tagged values for the next warp
  float *rq = reinterpret_cast<float *>(ring + (size_t)Z * kRing * 32);         // [Z][kQ][32] prefetched inputs
  int *prog = reinterpret_cast<int *>(rq + (size_t)Z * kQ * 32);              
  int *done = prog + Z;
  __shared__ int s_ticket, s_abort;
  if (threadIdx.x == 0) {
    s_ticket = atomicAdd(bm.ticket, 1);
    s_abort = 0;
  }
  for (int i = threadIdx.x; i < Z * kRing * 32; i += blockDim.x) ring[i] = ll_pack(0.f, 0x80000000u);
  if (threadIdx.x < Z) {
    prog[threadIdx.x] = INT_MAX;
    done[threadIdx.x] = INT_MAX;
  }
  __syncthreads();
  const int owner = owner_of(bm, s_ticket);
  const DevTet &t = tets[bm.order[owner]];
  const int ncta = bm.prefix[owner + 1] - bm.prefix[owner];
  const int cta = t.band.cta[ncta - 1 - (s_ticket - bm.prefix[owner])];  // reverse dependency order
  const int g = cta >> 16, k = cta & 0xffff;
  const int N = t.N;
  const int z = 1 + g * Z + wi;
    if (band_exists(N, z, k)) {
    const unsigned epoch = (unsigned)t.band.epoch[0];  // backward: even epochs
    const int KB = band_kmax(N) + 1;
    const BandInfo bi = t.band.info[(size_t)(z - 1) * KB + k];
    const int Y = band_Y(z, k), y = Y + lane;
    const bool row_ok = y >= 1 && y <= N - 2 - z;
    const int n = N - 1 - y - z;
    const int slo = band_slo(z, k), shi = band_shi(N, z, k);
    const bool have_up = band_exists(N, z + 1, k);
    const int slo_up = have_up ? band_slo(z + 1, k) : INT_MAX;  // the layer above writes steps >= slo_up
    float *wb = reinterpret_cast<float *>(t.band.w) + bi.off;
    unsigned long long *hs_out = t.band.streams + bi.hoff;  // lane 0 -> band k-1
    // the warp below in this CTA reads our ring; the bottom warp feeds the CTA below
    const bool bottom = wi == 0 || !band_exists(N, z - 1, k);
    unsigned long long *vs_out = nullptr;
    if (wi == 0 && z >= 2) vs_out = t.band.streams + t.band.info[(size_t)(z - 2) * KB + k].voff;
    // the warp above: ring of warp wi+1, or the CTA above through our layer's stream
    const bool top = wi == Z - 1 || z + 1 > N - 3;
    const unsigned long long *vs_in = (top && have_up) ? t.band.streams + bi.voff : nullptr;
    const bool need_n = row_ok && lane == 31 && band_exists(N, z, k + 1);      // n, nw from band k+1
    const bool need_t = row_ok && lane == 31 && band_exists(N, z + 1, k + 1);  // tc, tw from band k+1 above
    const bool has_edge = __shfl_sync(0xffffffffu, need_n || need_t, 31);
    const unsigned long long *hs_right = need_n ? t.band.streams + t.band.info[(size_t)(z - 1) * KB + k + 1].hoff : nullptr;
    const unsigned long long *hs_diag = need_t ? t.band.streams + t.band.info[(size_t)z * KB + k + 1].hoff : nullptr;
    Row8<(REG >= 0 ? REG : 0)> C;
    if (row_ok) C.template load<DXP>(reinterpret_cast<const float *>(t.tabB) + (size_t)row_id(N, y, z) * 8 * DXP);
    else C.zero();
    const float hh = (float)(0.5 * t.h);
    unsigned long long *my_ring = ring + (size_t)wi * kRing * 32;
    const unsigned long long *above_ring = !top ? ring + (size_t)(wi + 1) * kRing * 32 : nullptr;
    float *my_rq = rq + (size_t)wi * kQ * 32;

    auto prefetch = [&](int s) {
      if (s >= slo && s <= shi) {  // uniform
        cpa4_if(true, my_rq + (s & (kQ - 1)) * 32 + lane, wb + (size_t)(s - 1) * 32 + lane);
      }
      cpa_commit();
    };
    for (int s = shi; s > shi - kPre; --s) prefetch(s);
    // tagged words of step s-1, s-2 in flight (V: top warp; edges: lane 31,
    // which has no point before step 63)
    const ulonglong2 none2 = make_ulonglong2(0ull, 0ull);
    auto fetch_v = [&](int s) { return ld_ll_if(vs_in != nullptr && s >= slo_up && s >= slo, vs_in + (size_t)s * 32 + lane, 0ull); };
    auto fetch_r = [&](int s) { return ld_ll2_if(need_n && s >= 63 && s >= slo, hs_right + 2 * (s - 63), none2); };
    auto fetch_t = [&](int s) { return ld_ll2_if(need_t && s >= 63 && s >= slo, hs_diag + 2 * (s - 63), none2); };
    unsigned long long vq1 = fetch_v(shi), vq2 = fetch_v(shi - 1);
    ulonglong2 rq1 = fetch_r(shi), rq2 = fetch_r(shi - 1), tq1 = fetch_t(shi), tq2 = fetch_t(shi - 1);

    float v1 = 0.f, v2 = 0.f;  // this lane's values at steps s+1, s+2
    float u1 = 0.f, u2 = 0.f;  // layer above, this lane's column, steps s+1, s+2
    int cons_seen = INT_MAX;   // progress of the warp below (ring reuse)
    int above_seen = INT_MAX;  // progress of the warp above (ring fill)
    for (int s = shi; s >= slo; --s) {
      prefetch(s - kPre);
      cpa_wait<kPre>();
      const int slot = s & (kQ - 1);
      const int x = s - 2 * lane;
      const bool act = row_ok && x >= 1 && x <= n;
      // layer above, this lane's column at step s (none before the layer above starts)
      float u0 = 0.f;
      if (have_up && s >= slo_up) {  // uniform
        unsigned long long w;
        if (!top) {
          if (above_seen > s) {
            int v = INT_MAX;
            if (lane == 0) v = wait_hint(&done[wi + 1], s, false, &s_abort, status, max_spins, z, s);
            above_seen = __shfl_sync(0xffffffffu, v, 0);
            if (above_seen > s) break;  // gave up
          }
          u0 = ring_value(above_ring + (s & (kRing - 1)) * 32 + lane, (unsigned)s, &s_abort);
        } else {
          w = vq1;
          const bool ok = ll_tag(w) == epoch;
          if (!__all_sync(0xffffffffu, ok)) {
            if (!ok) w = ll_pack(poll_global(vs_in + (size_t)s * 32 + lane, epoch, &s_abort, status, max_spins, z, s), epoch);
            if (__shfl_sync(0xffffffffu, *(volatile int *)&s_abort, 0)) break;
          }
          u0 = ll_val(w);
        }
      }
      // neighbours in lane j+1; lane 31 takes them from band k+1 (edge words)
      float wn = __shfl_down_sync(0xffffffffu, v2, 1);   // (x, y+1, z)
      float wnw = __shfl_down_sync(0xffffffffu, v1, 1);  // (x-1, y+1, z)
      float wtc = __shfl_down_sync(0xffffffffu, u2, 1);  // (x, y, z+1)
      float wtw = __shfl_down_sync(0xffffffffu, u1, 1);  // (x-1, y, z+1)
      const bool inner = x + y + z <= N - 2;  // p-w, p-s, p-bc interior
      if (has_edge) {  // uniform: lane 31 of this warp needs band k+1
        unsigned long long e0 = rq1.x, e1 = rq1.y;
        unsigned long long e2 = tq1.x, e3 = tq1.y;
        // words read only where their term is used
        const bool u_nw = need_n && act && x >= 2, u_n = need_n && act && inner;
        const bool u_tw = need_t && act && x >= 2, u_tc = need_t && act && inner;
        const bool ok = (!u_nw || ll_tag(e0) == epoch) && (!u_n || ll_tag(e1) == epoch) &&
                        (!u_tw || ll_tag(e2) == epoch) && (!u_tc || ll_tag(e3) == epoch);
        if (!__all_sync(0xffffffffu, ok)) {
          if (!ok) {
            if (u_nw && ll_tag(e0) != epoch) e0 = ll_pack(poll_global(hs_right + 2 * (s - 63), epoch, &s_abort, status, max_spins, z, s), epoch);
            if (u_n && ll_tag(e1) != epoch) e1 = ll_pack(poll_global(hs_right + 2 * (s - 63) + 1, epoch, &s_abort, status, max_spins, z, s), epoch);
            if (u_tw && ll_tag(e2) != epoch) e2 = ll_pack(poll_global(hs_diag + 2 * (s - 63), epoch, &s_abort, status, max_spins, z, s), epoch);
            if (u_tc && ll_tag(e3) != epoch) e3 = ll_pack(poll_global(hs_diag + 2 * (s - 63) + 1, epoch, &s_abort, status, max_spins, z, s), epoch);
          }
          if (__shfl_sync(0xffffffffu, *(volatile int *)&s_abort, 0)) break;
        }
        if (lane == 31) {
          wnw = ll_val(e0);
          wn = ll_val(e1);
          wtw = ll_val(e2);
          wtc = ll_val(e3);
        }
      }
      // L[0] = 1/D~^p, L[1+d] = L~^{p-d}_d for d = w s se bnw bn bc be; every
      // lane evaluates, terms of neighbours outside the interior are selected away
      float L[8];
      C.eval((float)(2 * x - (N - y - z)) * hh, L);
      if constexpr (V1) {  // V1: stored exact 1/D^p at p and L^{p-d}_d where p - d is a cell-boundary point
        const float *bndv = reinterpret_cast<const float *>(t.bnd);
        if (bndv && act) {
          if (on_cell_boundary(N, x, y, z)) L[0] = bndv[(size_t)bnd_record(t.bnd_off, N, x, y, z) * 8 + 7];
#pragma unroll
          for (int d = 0; d < kNumLower; ++d) {
            const int qx = x - dir_dx(d), qy = y - dir_dy(d), qz = z - dir_dz(d);
            if (in_interior(N, qx, qy, qz) && on_cell_boundary(N, qx, qy, qz))
              L[1 + d] = bndv[(size_t)bnd_record(t.bnd_off, N, qx, qy, qz) * 8 + d];
          }
        }
      }
      const float zero = 0.f;
      wn = inner ? wn : zero;                                  // p - s   = (x, y+1, z)
      wtc = inner ? wtc : zero;                                // p - bc  = (x, y, z+1)
      const float wtse = (inner && y >= 2) ? u1 : zero;        // p - bnw = (x+1, y-1, z+1)
      wnw = x >= 2 ? wnw : zero;                               // p - se  = (x-1, y+1, z)
      wtw = x >= 2 ? wtw : zero;                               // p - be  = (x-1, y, z+1)
      const float wts = y >= 2 ? u0 : zero;                    // p - bn  = (x, y-1, z+1)
      const float we = inner ? v1 : zero;                      // p - w   = (x+1, y, z)
      float acc = L[0] * my_rq[slot * 32 + lane];
      acc = fmaf(-L[2], wn, acc);
      acc = fmaf(-L[6], wtc, acc);
      acc = fmaf(-L[4], wtse, acc);
      acc = fmaf(-L[3], wnw, acc);
      acc = fmaf(-L[7], wtw, acc);
      acc = fmaf(-L[5], wts, acc);
      acc = fmaf(-L[1], we, acc);
      const float val = act ? acc : zero;
      st_f32_if(act, wb + (size_t)(s - 1) * 32 + lane, val);
      if (bottom) {
        if (vs_out) st_ll_global(vs_out + (size_t)s * 32 + lane, ll_pack(val, epoch));
      } else {
        // the slot last held step s + kRing; the warp below reads steps from shi down
        if (s + kRing <= shi && cons_seen > s + kRing) {
          int seen = cons_seen;
          if (lane == 0) wait_progress(&prog[wi - 1], s + kRing, false, &s_abort, status, max_spins, z, s, &seen);
          cons_seen = __shfl_sync(0xffffffffu, seen, 0);
          if (cons_seen > s + kRing) break;  // gave up
        }
        st_ring(my_ring + (s & (kRing - 1)) * 32 + lane, ll_pack(val, (unsigned)s));
        st_hint_if(lane == 0, &done[wi], s);
      }
      st_ll2_if(lane == 0, hs_out + 2 * s, ll_pack(val, epoch), ll_pack(v1, epoch));  // record s
      st_hint_if(lane == 0 && !top, &prog[wi], s);
      v2 = v1;
      v1 = val;
      u2 = u1;
      u1 = u0;
      vq1 = vq2;
      vq2 = fetch_v(s - 2);
      rq1 = rq2;
      rq2 = fetch_r(s - 2);
      tq1 = tq2;
      tq2 = fetch_t(s - 2);
    }
    st_hint_if(lane == 0 && !top, &prog[wi], INT_MIN);
    // record slo - 1 = (none, value at slo): band k-1 needs its second half
    if (lane == 0 && !*(volatile int *)&s_abort) st_ll2_global(hs_out + 2 * (slo - 1), ll_pack(0.f, epoch), ll_pack(v1, epoch));
    cpa_wait<0>();
  }
}

// ------------------------------------------- residual / update (tiles) --

// residual at one interior point, operator from t (OP 0 constant stencil,
// 1 on-the-fly edge-star assembly, 2 stored coefficients); FP64 for double x
// starts of the seven grid rows a point's stencil touches (one row (y, z))
struct RowStarts {
  int64_t r0, rs, rn, rb, rbn, rt, rts;
};
__device__ __forceinline__ RowStarts row_starts(int N, int y, int z) {
  return {grid_index(N, 0, y, z),     grid_index(N, 0, y - 1, z), grid_index(N, 0, y + 1, z),
          grid_index(N, 0, y, z - 1), grid_index(N, 0, y + 1, z - 1), grid_index(N, 0, y, z + 1),
          grid_index(N, 0, y - 1, z + 1)};
}

template <typename TX, typename TR, int OP>
__device__ __forceinline__ TR residual_at(const DevTet &t, const TR *A15, const RowStarts &R, int x,
                                          const TX *__restrict__ xv_, const TX *__restrict__ b) {
  const int64_t r0 = R.r0, rs = R.rs, rn = R.rn, rb = R.rb, rbn = R.rbn, rt = R.rt, rts = R.rts;
  TR xv[15];
  xv[0] = (TR)xv_[r0 + x - 1];
  xv[1] = (TR)xv_[rs + x];
  xv[2] = (TR)xv_[rs + x + 1];
  xv[3] = (TR)xv_[rbn + x - 1];
  xv[4] = (TR)xv_[rbn + x];
  xv[5] = (TR)xv_[rb + x];
  xv[6] = (TR)xv_[rb + x + 1];
  xv[7] = (TR)xv_[r0 + x];
  xv[8] = (TR)xv_[r0 + x + 1];
  xv[9] = (TR)xv_[rn + x];
  xv[10] = (TR)xv_[rn + x - 1];
  xv[11] = (TR)xv_[rts + x + 1];
  xv[12] = (TR)xv_[rts + x];
  xv[13] = (TR)xv_[rt + x];
  xv[14] = (TR)xv_[rt + x - 1];
  TR res = (TR)b[r0 + x];
  if (OP == 0) {
#pragma unroll
    for (int d = 0; d < 15; ++d) res = fma(-A15[d], xv[d], res);
  } else if (OP == 2) {
    stored_apply(res, t.astore, t.astride, r0 + x, xv);
  } else {
    const double *kap = t.kappa;
    double kq[15];
    kq[0] = kap[r0 + x - 1];
    kq[1] = kap[rs + x];
    kq[2] = kap[rs + x + 1];
    kq[3] = kap[rbn + x - 1];
    kq[4] = kap[rbn + x];
    kq[5] = kap[rb + x];
    kq[6] = kap[rb + x + 1];
    kq[7] = kap[r0 + x];
    kq[8] = kap[r0 + x + 1];
    kq[9] = kap[rn + x];
    kq[10] = kap[rn + x - 1];
    kq[11] = kap[rts + x + 1];
    kq[12] = kap[rts + x];
    kq[13] = kap[rt + x];
    kq[14] = kap[rt + x - 1];
    star_apply_all(std::make_integer_sequence<int, 15>{}, res, kq, xv, t.Wstar);
  }
  return res;
}

// Tile = 32 steps of one band: each warp computes 4 rows along x (coalesced
// reads of x, b, kappa), the tile is transposed in shared memory and stored
// as 32 band lines.  MODE 0: r = b - A x (with the tile's ||r||^2), MODE 1:
// copy of a full-grid vector into the band array.  Four CTAs per SM (at most
// 64 registers): the kernel waits on its loads, and the extra warps halve its
// time at level 9 against two CTAs per SM.
template <typename TX, typename TR, int MODE>
__global__ void __launch_bounds__(256, 4) band_in_kernel(const DevTet *__restrict__ tets, const int *__restrict__ tprefix,
                                                      int ntets, const TX *const *__restrict__ xs,
                                                      const TX *const *__restrict__ bs, const TX *x1, const TX *b1,
                                                      double *__restrict__ partials) {
  __shared__ float T[32][33];
  __shared__ double red[8];
  int lo = 0, hi = ntets - 1;
  const int blk = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tprefix[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  const DevTet &t = tets[lo];
  const int N = t.N;
  const int tile = t.band.tiles[blk - tprefix[lo]];
  const int z = tile >> 20, k = (tile >> 14) & 63, c = tile & 16383;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (blk == tprefix[lo] && threadIdx.x == 0) t.band.epoch[0] += 2;  // new epochs for this sweep's substitutions
  const int Y = band_Y(z, k);
  const int s0 = 1 + 32 * c;
  const TX *xv = xs ? xs[lo] : x1;
  const TX *b = bs ? bs[lo] : b1;
  const int op = t.const_kappa ? 0 : (t.astore ? 2 : 1);
  // the constant stencil, converted once per block to the residual type
  __shared__ TR sA15[15];
  if (threadIdx.x < 15) sA15[threadIdx.x] = (TR)t.A15[threadIdx.x];
  __syncthreads();
  double acc2 = 0.0;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int j = warp + 8 * m, y = Y + j;
    const int x = s0 + lane - 2 * j;
    TR r = 0;
    if (y >= 1 && y <= N - 2 - z) {  // warp-uniform: the row's starts once per row
      const RowStarts R = row_starts(N, y, z);
      if (x >= 1 && x <= N - 1 - y - z) {
        if (MODE == 0)
          r = op == 0 ? residual_at<TX, TR, 0>(t, sA15, R, x, xv, b)
                      : (op == 2 ? residual_at<TX, TR, 2>(t, sA15, R, x, xv, b)
                                 : residual_at<TX, TR, 1>(t, sA15, R, x, xv, b));
        else r = (TR)xv[R.r0 + x];
        acc2 += (double)r * (double)r;
      }
    }
    T[lane][j] = (float)r;
  }
  __syncthreads();
  const int shi = band_shi(N, z, k);
  float *wb = reinterpret_cast<float *>(t.band.w) + t.band.info[(size_t)(z - 1) * (band_kmax(N) + 1) + k].off;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int sl = warp + 8 * m;
    if (s0 + sl <= shi) wb[(size_t)(s0 + sl - 1) * 32 + lane] = T[sl][lane];
  }
  if (MODE == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
    if (lane == 0) red[warp] = acc2;
    __syncthreads();
    if (threadIdx.x == 0 && partials) {
      double sum = 0.0;
      for (int i = 0; i < 8; ++i) sum += red[i];
      partials[blk] = sum;
    }
  }
}

// x += w (band array -> full grid), through the same tiles
template <typename TX>
__global__ void __launch_bounds__(256) band_update_kernel(const DevTet *__restrict__ tets, const int *__restrict__ tprefix,
                                                          int ntets, TX *const *__restrict__ xs, TX *x1) {
  __shared__ float T[32][33];
  int lo = 0, hi = ntets - 1;
  const int blk = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tprefix[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  const DevTet &t = tets[lo];
  const int N = t.N;
  const int tile = t.band.tiles[blk - tprefix[lo]];
  const int z = tile >> 20, k = (tile >> 14) & 63, c = tile & 16383;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Y = band_Y(z, k);
  const int s0 = 1 + 32 * c;
  const int shi = band_shi(N, z, k);
  const float *wb = reinterpret_cast<const float *>(t.band.w) + t.band.info[(size_t)(z - 1) * (band_kmax(N) + 1) + k].off;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int sl = warp + 8 * m;
    T[sl][lane] = s0 + sl <= shi ? wb[(size_t)(s0 + sl - 1) * 32 + lane] : 0.f;
  }
  __syncthreads();
  TX *xv = xs ? xs[lo] : x1;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int j = warp + 8 * m, y = Y + j;
    const int x = s0 + lane - 2 * j;
    if (y >= 1 && y <= N - 2 - z) {
      const int64_t r0 = grid_index(N, 0, y, z);
      if (x >= 1 && x <= N - 1 - y - z) xv[r0 + x] = xv[r0 + x] + (TX)T[lane][j];
    }
  }
}

template <int DXP, int REG, bool V1>
cudaError_t launch_fb1(bool fwd, const BandLaunch &L, LaunchStatus *status, long long max_spins, cudaStream_t st) {
  auto kernel = fwd ? fwd_band<DXP, REG, V1> : bwd_band<DXP, REG, V1>;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_smem_bytes(8));
  if (e != cudaSuccess) return e;
  kernel<<<L.ctas, L.Z * 32, band_smem_bytes(L.Z), st>>>(L.tets, fwd ? L.map_f : L.map_b, status, max_spins);
  return cudaGetLastError();
}
template <int DXP, int REG>
cudaError_t launch_fb(bool fwd, const BandLaunch &L, LaunchStatus *status, long long max_spins, cudaStream_t st) {
  return L.v1 ? launch_fb1<DXP, REG, true>(fwd, L, status, max_spins, st)
              : launch_fb1<DXP, REG, false>(fwd, L, status, max_spins, st);
}

}  // namespace

size_t band_smem_bytes(int Z) {
  return (size_t)Z * kRing * 32 * 8 + (size_t)Z * kQ * 32 * 4 + Z * 8;
}

cudaError_t launch_band_sub(bool forward, const BandLaunch &L, LaunchStatus *status, long long max_spins,
                            cudaStream_t st) {
  if (L.Z < 1 || L.Z > 8) return cudaErrorInvalidValue;
  switch (L.reg) {
    case 0: return launch_fb<4, 0>(forward, L, status, max_spins, st);
    case 1: return launch_fb<4, 1>(forward, L, status, max_spins, st);
    case 2: return launch_fb<4, 2>(forward, L, status, max_spins, st);
    case 3: return launch_fb<4, 3>(forward, L, status, max_spins, st);
    case 4: return launch_fb<8, 4>(forward, L, status, max_spins, st);
    case 5: return launch_fb<8, 5>(forward, L, status, max_spins, st);
    case 6: return launch_fb<8, 6>(forward, L, status, max_spins, st);
    case 7: return launch_fb<8, 7>(forward, L, status, max_spins, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_band_in(int kind, int mode, const DevTet *tets, const int *tprefix, int ntets, int total_tiles,
                           const void *const *xs, const void *const *bs, const void *x1, const void *b1,
                           double *partials, cudaStream_t st) {
  if (total_tiles <= 0) return cudaSuccess;
  if (kind == kSweepF32) {
    using T = float;
    auto X = reinterpret_cast<const T *const *>(xs);
    auto B = reinterpret_cast<const T *const *>(bs);
    auto X1 = reinterpret_cast<const T *>(x1);
    auto B1 = reinterpret_cast<const T *>(b1);
    if (mode == 0) band_in_kernel<T, T, 0><<<total_tiles, 256, 0, st>>>(tets, tprefix, ntets, X, B, X1, B1, partials);
    else band_in_kernel<T, T, 1><<<total_tiles, 256, 0, st>>>(tets, tprefix, ntets, X, B, X1, B1, partials);
  } else {
    using T = double;
    auto X = reinterpret_cast<const T *const *>(xs);
    auto B = reinterpret_cast<const T *const *>(bs);
    auto X1 = reinterpret_cast<const T *>(x1);
    auto B1 = reinterpret_cast<const T *>(b1);
    if (mode == 0) band_in_kernel<T, T, 0><<<total_tiles, 256, 0, st>>>(tets, tprefix, ntets, X, B, X1, B1, partials);
    else band_in_kernel<T, T, 1><<<total_tiles, 256, 0, st>>>(tets, tprefix, ntets, X, B, X1, B1, partials);
  }
  return cudaGetLastError();
}

cudaError_t launch_band_update(int kind, const DevTet *tets, const int *tprefix, int ntets, int total_tiles,
                               void *const *xs, void *x1, cudaStream_t st) {
  if (total_tiles <= 0) return cudaSuccess;
  if (kind == kSweepF32)
    band_update_kernel<float><<<total_tiles, 256, 0, st>>>(tets, tprefix, ntets, reinterpret_cast<float *const *>(xs),
                                                           reinterpret_cast<float *>(x1));
  else
    band_update_kernel<double><<<total_tiles, 256, 0, st>>>(tets, tprefix, ntets,
                                                            reinterpret_cast<double *const *>(xs),
                                                            reinterpret_cast<double *>(x1));
  return cudaGetLastError();
}

}  // namespace ilu
