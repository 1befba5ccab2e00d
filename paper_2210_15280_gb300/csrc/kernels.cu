// kernels.cu -- sweep kernels of the matrix-free surrogate ILU(0) smoother
// (arXiv 2210.15280, Alg. 2, V2 boundary rule) for sm_103a.
//
// One sweep is three launches:
//   residual   r = b - A x on every interior point, fully parallel (one warp
//              per grid row, coalesced along x); the operator is the constant
//              15-point stencil or is assembled on the fly from kappa at the
//              grid points (edge-star weights); FP64 for F64/MIXED.
//   forward    w = L~^{-1} r  (in place), level-scheduled on the hyperplanes
//              x + 2y + 3z = s: every lower direction has a negative hyperplane
//              weight, so the points of one level are independent.
//   backward   w = L~^{-T} D~^{-1} w, x += w, the same levels in reverse.
// The wavefront kernels split the tet into z-slabs, one CTA per slab and one
// warp per face layer.  The last three levels of w of the slab stay in a
// shared-memory ring; the layer just outside the slab is read from global
// memory after the neighbouring slab has published its progress.  CTAs take
// slab numbers from an atomic ticket in dependency order, so a CTA only ever
// waits for CTAs that are already running; every wait is bounded.
#include <cuda_runtime.h>

#include <climits>
#include <utility>

#include "kernels.cuh"

namespace ilu {

namespace {

// ------------------------------------------- edge-star pattern (unrolled) --

template <int E>
__device__ __forceinline__ void star_term(double *A, const double *kq, const double *W) {
  constexpr int D = star_d(E);
  constexpr int Q = star_q(E);
  A[D] = fma(W[E], kq[Q], A[D]);
}
template <int... E>
__device__ __forceinline__ void star_all(std::integer_sequence<int, E...>, double *A, const double *kq,
                                         const double *W) {
  (star_term<E>(A, kq, W), ...);
}

// --------------------------------------------------------- small helpers --

__device__ __forceinline__ int ylo_of(int N, int s, int z) { return max(1, s - 2 * z - N + 1); }
__device__ __forceinline__ int yhi_of(int s, int z) {
  const int v = s - 3 * z - 1;
  return v < 0 ? 0 : v >> 1;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T horner(const T *c, int n, T t) {
  T v = c[n];
  for (int k = n - 1; k >= 0; --k) v = fma(v, t, c[k]);
  return v;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T *p) {
  return __ldcg(p);
}

// Bounded wait of thread 0 for flags[idx] >= target.  Returns false on timeout.
__device__ bool wait_flag(const int *flag, int target, int &seen, long long max_spins) {
  if (seen >= target) return true;
  long long spins = 0;
  int v = ld_acquire(flag);
  while (v < target) {
    if (++spins > max_spins) return false;
    __nanosleep(32);
    v = ld_acquire(flag);
  }
  seen = v;
  return true;
}

// --------------------------------------------------------------- residual --

// r = b - A x at interior points of rows (y, z); one warp per row.
template <typename TX, typename TR, typename TW, bool VAR>
__global__ void __launch_bounds__(256) residual_kernel(DevTet t, const TX *__restrict__ x,
                                                       const TX *__restrict__ b, TW *__restrict__ r,
                                                       double *__restrict__ partials) {
  const int N = t.N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int z = blockIdx.y + 1;
  const int y = blockIdx.x * 8 + warp + 1;
  double acc2 = 0.0;
  if (y + z <= N - 2) {
    const int n = N - 1 - y - z;
    // row starts of the seven rows the stencil touches
    const int64_t r0 = grid_index(N, 0, y, z);          // (y, z)
    const int64_t rs = grid_index(N, 0, y - 1, z);      // (y-1, z)
    const int64_t rn = grid_index(N, 0, y + 1, z);      // (y+1, z)
    const int64_t rb = grid_index(N, 0, y, z - 1);      // (y, z-1)
    const int64_t rbn = grid_index(N, 0, y + 1, z - 1); // (y+1, z-1)
    const int64_t rt = grid_index(N, 0, y, z + 1);      // (y, z+1)
    const int64_t rts = grid_index(N, 0, y - 1, z + 1); // (y-1, z+1)
    for (int xx = 1 + lane; xx <= n; xx += 32) {
      // neighbour values in the order of D: w s se bnw bn bc be c e n nw tse ts tc tw
      TR xv[15];
      xv[0] = (TR)x[r0 + xx - 1];
      xv[1] = (TR)x[rs + xx];
      xv[2] = (TR)x[rs + xx + 1];
      xv[3] = (TR)x[rbn + xx - 1];
      xv[4] = (TR)x[rbn + xx];
      xv[5] = (TR)x[rb + xx];
      xv[6] = (TR)x[rb + xx + 1];
      xv[7] = (TR)x[r0 + xx];
      xv[8] = (TR)x[r0 + xx + 1];
      xv[9] = (TR)x[rn + xx];
      xv[10] = (TR)x[rn + xx - 1];
      xv[11] = (TR)x[rts + xx + 1];
      xv[12] = (TR)x[rts + xx];
      xv[13] = (TR)x[rt + xx];
      xv[14] = (TR)x[rt + xx - 1];
      TR res = (TR)b[r0 + xx];
      if (!VAR) {
#pragma unroll
        for (int d = 0; d < 15; ++d) res = fma(-(TR)t.A15[d], xv[d], res);
      } else {
        const double *kap = t.kappa;
        double kq[15];
        kq[0] = kap[r0 + xx - 1];
        kq[1] = kap[rs + xx];
        kq[2] = kap[rs + xx + 1];
        kq[3] = kap[rbn + xx - 1];
        kq[4] = kap[rbn + xx];
        kq[5] = kap[rb + xx];
        kq[6] = kap[rb + xx + 1];
        kq[7] = kap[r0 + xx];
        kq[8] = kap[r0 + xx + 1];
        kq[9] = kap[rn + xx];
        kq[10] = kap[rn + xx - 1];
        kq[11] = kap[rts + xx + 1];
        kq[12] = kap[rts + xx];
        kq[13] = kap[rt + xx];
        kq[14] = kap[rt + xx - 1];
        double A[15];
#pragma unroll
        for (int d = 0; d < 15; ++d) A[d] = 0.0;
        star_all(std::make_integer_sequence<int, 100>{}, A, kq, t.Wstar);
        // rows sum to zero: (A x)_p = sum_{d != c} A_d (x_{p+d} - x_p)
        const double xc = (double)xv[7];
#pragma unroll
        for (int d = 0; d < 15; ++d)
          if (d != 7) res = (TR)fma(-A[d], (double)xv[d] - xc, (double)res);
      }
      r[r0 + xx] = (TW)res;
      acc2 += (double)res * (double)res;
    }
  }
  // deterministic block reduction of the squared norm
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  __shared__ double red[8];
  if (lane == 0) red[warp] = acc2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k];
    partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void norm_finish_kernel(const double *__restrict__ partials, int n, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(red[0]);
}

// ---------------------------------------------------------------- forward --

// In-place forward substitution w <- L~^{-1} w for the interior of one tet.
template <typename TW>
__global__ void __launch_bounds__(1024) forward_kernel(DevTet t, LaunchStatus *status, long long max_spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TW *ring = reinterpret_cast<TW *>(smem_raw);
  __shared__ int s_slab, s_abort;
  const int N = t.N, Zb = t.slab_layers, P = t.nslabs;
  const int RC = N / 2 + 2;
  int *flags = t.flags;
  if (threadIdx.x == 0) {
    s_slab = atomicAdd(&flags[2 * P], 1);
    s_abort = 0;
  }
  __syncthreads();
  const int k = s_slab;
  if (k >= P) return;
  const int zs = 1 + k * Zb, ze = min(zs + Zb, N - 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int z = zs + warp;
  const bool active = z < ze;
  const int s_begin = 3 * zs + 3, s_end = 2 * N + ze - 4;
  const TW *tab = reinterpret_cast<const TW *>(t.tabF);
  TW *wg = reinterpret_cast<TW *>(t.w);
  const int S = t.rstride, dxg = t.dx;
  const TW hh = (TW)(0.5 * t.h);
  int seen = 0;
  if (threadIdx.x == 0 && k > 0) {
    if (!wait_flag(&flags[k - 1], s_begin, seen, max_spins)) {
      s_abort = 1;
      atomicCAS(&status->code, 0, 6);
      status->where = k;
      status->level = s_begin;
    }
  }
  __syncthreads();
  for (int s = s_begin; s <= s_end && !s_abort; ++s) {
    if (active) {
      const int ylo = ylo_of(N, s, z), yhi = yhi_of(s, z);
      TW *slot = ring + ((size_t)(s & 3) * Zb + warp) * RC;
      const TW *m1 = ring + ((size_t)((s - 1) & 3) * Zb + warp) * RC;
      const TW *m2 = ring + ((size_t)((s - 2) & 3) * Zb + warp) * RC;
      const bool halo = (warp == 0);  // layer z-1 belongs to the previous slab
      const TW *b1 = halo ? nullptr : ring + ((size_t)((s - 1) & 3) * Zb + warp - 1) * RC;
      const TW *b2 = halo ? nullptr : ring + ((size_t)((s - 2) & 3) * Zb + warp - 1) * RC;
      const TW *b3 = halo ? nullptr : ring + ((size_t)((s - 3) & 3) * Zb + warp - 1) * RC;
      const int ylo1 = ylo_of(N, s - 1, z), ylo2 = ylo_of(N, s - 2, z);
      const int zl1 = ylo_of(N, s - 1, z - 1), zl2 = ylo_of(N, s - 2, z - 1), zl3 = ylo_of(N, s - 3, z - 1);
      for (int y = ylo + lane; y <= yhi; y += 32) {
        const int x = s - 2 * y - 3 * z;
        const int64_t gi = grid_index(N, x, y, z);
        const TW *c = tab + (size_t)row_id(N, y, z) * 7 * S;
        const TW tt = (TW)(2 * x - (N - y - z)) * hh;
        TW acc = wg[gi];
        if (x >= 2) acc = fma(-horner(c + 0 * S, dxg, tt), m1[y - ylo1], acc);
        if (y >= 2) {
          acc = fma(-horner(c + 1 * S, dxg, tt), m2[y - 1 - ylo2], acc);
          acc = fma(-horner(c + 2 * S, dxg, tt), m1[y - 1 - ylo1], acc);
        }
        if (z >= 2) {
          TW vbnw = 0, vbn, vbc, vbe;
          if (halo) {
            if (x >= 2) vbnw = ldcg(wg + grid_index(N, x - 1, y + 1, z - 1));
            vbn = ldcg(wg + grid_index(N, x, y + 1, z - 1));
            vbc = ldcg(wg + grid_index(N, x, y, z - 1));
            vbe = ldcg(wg + grid_index(N, x + 1, y, z - 1));
          } else {
            if (x >= 2) vbnw = b2[y + 1 - zl2];
            vbn = b1[y + 1 - zl1];
            vbc = b3[y - zl3];
            vbe = b2[y - zl2];
          }
          if (x >= 2) acc = fma(-horner(c + 3 * S, dxg, tt), vbnw, acc);
          acc = fma(-horner(c + 4 * S, dxg, tt), vbn, acc);
          acc = fma(-horner(c + 5 * S, dxg, tt), vbc, acc);
          acc = fma(-horner(c + 6 * S, dxg, tt), vbe, acc);
        }
        slot[y - ylo] = acc;
        wg[gi] = acc;
      }
    }
    if (threadIdx.x == 0) {
      if (k + 1 < P) {
        __threadfence();
        st_release(&flags[k], s);  // levels <= s-1 complete (barrier of the previous iteration)
      }
      if (k > 0 && s < s_end && !wait_flag(&flags[k - 1], s + 1, seen, max_spins)) {
        s_abort = 1;
        atomicCAS(&status->code, 0, 6);
        status->where = k;
        status->level = s + 1;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && k + 1 < P) {
    __threadfence();
    st_release(&flags[k], INT_MAX / 2);
  }
}

// --------------------------------------------------------------- backward --

// w <- D~^{-1} w - sum_d L~^{p-d}_d w^{p-d} in reverse level order, x += w.
template <typename TW, typename TX>
__global__ void __launch_bounds__(1024) backward_kernel(DevTet t, TX *__restrict__ xg, LaunchStatus *status,
                                                        long long max_spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TW *ring = reinterpret_cast<TW *>(smem_raw);
  __shared__ int s_slab, s_abort;
  const int N = t.N, Zb = t.slab_layers, P = t.nslabs;
  const int RC = N / 2 + 2;
  int *flags = t.flags + P;  // backward progress words
  if (threadIdx.x == 0) {
    s_slab = P - 1 - atomicAdd(&t.flags[2 * P + 1], 1);
    s_abort = 0;
  }
  __syncthreads();
  const int k = s_slab;
  if (k < 0) return;
  const int zs = 1 + k * Zb, ze = min(zs + Zb, N - 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int z = zs + warp;
  const bool active = z < ze;
  const int s_begin = 3 * zs + 3, s_end = 2 * N + ze - 4;
  const int TOP = 3 * N + 1;  // progress value for "level s done" is TOP - s
  const TW *tab = reinterpret_cast<const TW *>(t.tabB);
  TW *wg = reinterpret_cast<TW *>(t.w);
  const int S = t.rstride, dxg = t.dx;
  const TW hh = (TW)(0.5 * t.h);
  int seen = 0;
  if (threadIdx.x == 0 && k + 1 < P) {
    if (!wait_flag(&flags[k + 1], TOP - (s_end + 1), seen, max_spins)) {
      s_abort = 1;
      atomicCAS(&status->code, 0, 6);
      status->where = k;
      status->level = s_end;
    }
  }
  __syncthreads();
  for (int s = s_end; s >= s_begin && !s_abort; --s) {
    if (active) {
      const int ylo = ylo_of(N, s, z), yhi = yhi_of(s, z);
      TW *slot = ring + ((size_t)(s & 3) * Zb + warp) * RC;
      const TW *p1 = ring + ((size_t)((s + 1) & 3) * Zb + warp) * RC;
      const TW *p2 = ring + ((size_t)((s + 2) & 3) * Zb + warp) * RC;
      const bool halo = (warp == Zb - 1) || (z + 1 >= ze);  // layer z+1 belongs to the next slab
      const TW *u1 = halo ? nullptr : ring + ((size_t)((s + 1) & 3) * Zb + warp + 1) * RC;
      const TW *u2 = halo ? nullptr : ring + ((size_t)((s + 2) & 3) * Zb + warp + 1) * RC;
      const TW *u3 = halo ? nullptr : ring + ((size_t)((s + 3) & 3) * Zb + warp + 1) * RC;
      const int ylo1 = ylo_of(N, s + 1, z), ylo2 = ylo_of(N, s + 2, z);
      const int zl1 = ylo_of(N, s + 1, z + 1), zl2 = ylo_of(N, s + 2, z + 1), zl3 = ylo_of(N, s + 3, z + 1);
      for (int y = ylo + lane; y <= yhi; y += 32) {
        const int x = s - 2 * y - 3 * z;
        const int64_t gi = grid_index(N, x, y, z);
        const TW *c = tab + (size_t)row_id(N, y, z) * 8 * S;
        const TW tt = (TW)(2 * x - (N - y - z)) * hh;
        TW acc = horner(c, dxg, tt) * wg[gi];
        const bool inner = x + y + z <= N - 2;  // p - w, p - s, p - bc interior
        if (inner) {
          acc = fma(-horner(c + 1 * S, dxg, tt), p1[y - ylo1], acc);        // p - w  = (x+1, y, z)
          acc = fma(-horner(c + 2 * S, dxg, tt), p2[y + 1 - ylo2], acc);    // p - s  = (x, y+1, z)
        }
        if (x >= 2) acc = fma(-horner(c + 3 * S, dxg, tt), p1[y + 1 - ylo1], acc);  // p - se = (x-1, y+1, z)
        // upper layer z+1
        TW vbnw = 0, vbn = 0, vbc = 0, vbe = 0;
        const bool has_bnw = (y >= 2) && inner, has_bn = (y >= 2), has_bc = inner, has_be = (x >= 2);
        if (halo) {
          if (has_bnw) vbnw = ldcg(wg + grid_index(N, x + 1, y - 1, z + 1));
          if (has_bn) vbn = ldcg(wg + grid_index(N, x, y - 1, z + 1));
          if (has_bc) vbc = ldcg(wg + grid_index(N, x, y, z + 1));
          if (has_be) vbe = ldcg(wg + grid_index(N, x - 1, y, z + 1));
        } else {
          if (has_bnw) vbnw = u2[y - 1 - zl2];
          if (has_bn) vbn = u1[y - 1 - zl1];
          if (has_bc) vbc = u3[y - zl3];
          if (has_be) vbe = u2[y - zl2];
        }
        if (has_bnw) acc = fma(-horner(c + 4 * S, dxg, tt), vbnw, acc);
        if (has_bn) acc = fma(-horner(c + 5 * S, dxg, tt), vbn, acc);
        if (has_bc) acc = fma(-horner(c + 6 * S, dxg, tt), vbc, acc);
        if (has_be) acc = fma(-horner(c + 7 * S, dxg, tt), vbe, acc);
        slot[y - ylo] = acc;
        wg[gi] = acc;
        xg[gi] = xg[gi] + (TX)acc;
      }
    }
    if (threadIdx.x == 0) {
      if (k > 0) {
        __threadfence();
        st_release(&flags[k], TOP - (s + 1));  // levels >= s+1 complete
      }
      if (k + 1 < P && s > s_begin && !wait_flag(&flags[k + 1], TOP - s, seen, max_spins)) {
        s_abort = 1;
        atomicCAS(&status->code, 0, 6);
        status->where = k;
        status->level = s - 1;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && k > 0) {
    __threadfence();
    st_release(&flags[k], INT_MAX / 2);
  }
}

}  // namespace

// ------------------------------------------------------------ launchers --

int residual_blocks(int N) { return ((N - 3 + 7) / 8) * (N - 3); }

size_t sweep_smem_bytes(int N, int slab_layers, int kind) {
  const size_t e = kind == kSweepF64 ? sizeof(double) : sizeof(float);
  return (size_t)4 * slab_layers * (N / 2 + 2) * e;
}

cudaError_t launch_residual(const DevTet &t, int kind, const void *x, const void *b, void *r_out, double *partials,
                            int nblocks_cap, int *nblocks_used, cudaStream_t st) {
  const int N = t.N;
  dim3 grid((N - 3 + 7) / 8, N - 3);
  if ((int)(grid.x * grid.y) > nblocks_cap) return cudaErrorInvalidValue;
  if (nblocks_used) *nblocks_used = grid.x * grid.y;
  const bool var = !t.const_kappa;
  if (kind == kSweepF64) {
    if (var)
      residual_kernel<double, double, double, true><<<grid, 256, 0, st>>>(t, (const double *)x, (const double *)b,
                                                                            (double *)r_out, partials);
    else
      residual_kernel<double, double, double, false><<<grid, 256, 0, st>>>(t, (const double *)x, (const double *)b,
                                                                             (double *)r_out, partials);
  } else if (kind == kSweepMixed) {
    if (var)
      residual_kernel<double, double, float, true><<<grid, 256, 0, st>>>(t, (const double *)x, (const double *)b,
                                                                           (float *)r_out, partials);
    else
      residual_kernel<double, double, float, false><<<grid, 256, 0, st>>>(t, (const double *)x, (const double *)b,
                                                                            (float *)r_out, partials);
  } else {
    if (var)
      residual_kernel<float, float, float, true><<<grid, 256, 0, st>>>(t, (const float *)x, (const float *)b,
                                                                         (float *)r_out, partials);
    else
      residual_kernel<float, float, float, false><<<grid, 256, 0, st>>>(t, (const float *)x, (const float *)b,
                                                                          (float *)r_out, partials);
  }
  return cudaGetLastError();
}

cudaError_t launch_norm_finish(const double *partials, int n, double *out, cudaStream_t st) {
  norm_finish_kernel<<<1, 256, 0, st>>>(partials, n, out);
  return cudaGetLastError();
}

template <typename TW>
static cudaError_t fwd_impl(const DevTet &t, LaunchStatus *status, long long max_spins, cudaStream_t st) {
  const size_t smem = (size_t)4 * t.slab_layers * (t.N / 2 + 2) * sizeof(TW);
  cudaError_t e = cudaFuncSetAttribute(forward_kernel<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  forward_kernel<TW><<<t.nslabs, 32 * t.slab_layers, smem, st>>>(t, status, max_spins);
  return cudaGetLastError();
}

template <typename TW, typename TX>
static cudaError_t bwd_impl(const DevTet &t, void *x, LaunchStatus *status, long long max_spins, cudaStream_t st) {
  const size_t smem = (size_t)4 * t.slab_layers * (t.N / 2 + 2) * sizeof(TW);
  cudaError_t e =
      cudaFuncSetAttribute(backward_kernel<TW, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  backward_kernel<TW, TX><<<t.nslabs, 32 * t.slab_layers, smem, st>>>(t, (TX *)x, status, max_spins);
  return cudaGetLastError();
}

cudaError_t launch_forward(const DevTet &t, int kind, LaunchStatus *status, long long max_spins, cudaStream_t st) {
  if (kind == kSweepF64) return fwd_impl<double>(t, status, max_spins, st);
  return fwd_impl<float>(t, status, max_spins, st);
}

cudaError_t launch_backward(const DevTet &t, int kind, void *x, LaunchStatus *status, long long max_spins,
                            cudaStream_t st) {
  if (kind == kSweepF64) return bwd_impl<double, double>(t, x, status, max_spins, st);
  if (kind == kSweepMixed) return bwd_impl<float, double>(t, x, status, max_spins, st);
  return bwd_impl<float, float>(t, x, status, max_spins, st);
}

}  // namespace ilu
