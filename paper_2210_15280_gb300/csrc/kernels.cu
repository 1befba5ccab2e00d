// kernels.cu -- sweep kernels of the matrix-free surrogate ILU(0) smoother
// (arXiv 2210.15280, Alg. 2, V2 boundary rule) for sm_103a.
//
// One sweep is three launches: this file holds the first,
//   residual   r = b - A x on every interior point, fully parallel (one warp
//              per grid row, coalesced along x); the operator is the constant
//              15-point stencil or is assembled on the fly from kappa at the
//              grid points (edge-star weights); FP64 for F64/MIXED,
// and the deterministic norm reduction; wavefront.cu holds the forward and
// backward substitutions.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <type_traits>
#include <utility>

#include "kernels.cuh"
#include "packed.h"
#include "stencil.cuh"

namespace ilu {

namespace {

// --------------------------------------------------------- small helpers --

// --------------------------------------------------------------- residual --

// Where a row's operator comes from: the constant stencil, or the edge-star
// weights and kappa at the grid points, or the stored coefficients.
struct StencilData {
  const void *A15;     // the constant stencil in the residual type (a per-block copy)
  const double *Wstar, *kappa;
  const void *astore;  // stored off-diagonal coefficients (MODE 2)
  int64_t astride;
};

// MODE of the operator (kernels.cuh): constant stencil, assembled on the fly
// from kappa, or stored coefficients (the same values as on the fly)

// r = b - A x at the interior points x0 + lane of row (y, z) (one warp, one
// 32-point chunk of the row); returns this lane's share of ||r||^2
// (pmap non-null: r goes to the packed array pw instead, at the slot of the
// point's row, pmap[row id] = forward first step | lane << 20)
template <typename TX, typename TR, typename TW, int MODE>
__device__ __forceinline__ double residual_chunk(const StencilData &t, int N, int y, int z, int x0, int lane,
                                                 const TX *__restrict__ x, const TX *__restrict__ b,
                                                 TW *__restrict__ r, const int *__restrict__ pmap = nullptr,
                                                 float *__restrict__ pw = nullptr) {
  double acc2 = 0.0;
  if (y + z > N - 2) return acc2;
  const int n = N - 1 - y - z;
  // row starts of the seven rows the stencil touches
  const int64_t r0 = grid_index(N, 0, y, z);          // (y, z)
  const int64_t rs = grid_index(N, 0, y - 1, z);      // (y-1, z)
  const int64_t rn = grid_index(N, 0, y + 1, z);      // (y+1, z)
  const int64_t rb = grid_index(N, 0, y, z - 1);      // (y, z-1)
  const int64_t rbn = grid_index(N, 0, y + 1, z - 1); // (y+1, z-1)
  const int64_t rt = grid_index(N, 0, y, z + 1);      // (y, z+1)
  const int64_t rts = grid_index(N, 0, y - 1, z + 1); // (y-1, z+1)
  {
    const int xx = x0 + lane;
    if (xx > n) return acc2;
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
    if (MODE == kOpConst) {
      const TR *A15 = static_cast<const TR *>(t.A15);
#pragma unroll
      for (int d = 0; d < 15; ++d) res = fma(-A15[d], xv[d], res);
    } else if (MODE == kOpStored) {
      stored_apply(res, t.astore, t.astride, r0 + xx, xv);
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
      star_apply_all(std::make_integer_sequence<int, 15>{}, res, kq, xv, t.Wstar);
    }
    if (pmap) {
      const int m = pmap[row_id(N, y, z)];
      pw[packed_index((m & 0xfffff) + xx - 1, m >> 20)] = (float)res;
    } else {
      r[r0 + xx] = (TW)res;
    }
    acc2 += (double)res * (double)res;
  }
  return acc2;
}

// One tet: a warp per kResidualCPW consecutive 32-point chunks of interior
// rows (the chunk list balances rows of every length), 8 warps per block,
// per-block partial norms.
template <typename TX, typename TR, typename TW, int MODE>
__global__ void __launch_bounds__(256, MODE == kOpStar ? 1 : 4) residual_kernel(DevTet t, const TX *__restrict__ x,
                                                       const TX *__restrict__ b, TW *__restrict__ r,
                                                       double *__restrict__ partials, bool packed) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the constant stencil, converted once per block to the residual type
  __shared__ TR sA15[15];
  if (threadIdx.x < 15) sA15[threadIdx.x] = (TR)t.A15[threadIdx.x];
  __syncthreads();
  const StencilData sd{sA15, t.Wstar, t.kappa, t.astore, t.astride};
  double acc2 = 0.0;
  const int c0 = (blockIdx.x * 8 + warp) * kResidualCPW;  // this warp's consecutive chunks
#pragma unroll 1
  for (int k = 0; k < kResidualCPW && c0 + k < t.nchunks; ++k) {
    const int ch = t.chunks[c0 + k];
    acc2 += residual_chunk<TX, TR, TW, MODE>(sd, t.N, (ch >> 10) & 1023, ch >> 20, 1 + 32 * (ch & 1023), lane, x, b,
                                             r, packed ? t.pk.row_map : nullptr, packed ? t.pk.pw : nullptr);
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
    partials[blockIdx.x] = s;
  }
}

// Many tets whose operators come the same way (MODE): 1-D grid, tet
// order[i] owns blocks [bprefix[i], bprefix[i+1]) laid out as its single-tet
// grid; the result goes to the tet's packed array if it has one, else to its
// scratch w.  One launch per operator kind keeps the register count of each
// kernel that of its own arithmetic.
template <typename TX, typename TR, typename TW, int MODE>
__global__ void __launch_bounds__(256, MODE == kOpStar ? 1 : 4)
    residual_batch_kernel(const DevTet *__restrict__ tets, const int *__restrict__ order,
                          const int *__restrict__ bprefix, int n, const TX *const *__restrict__ xs,
                          const TX *const *__restrict__ bs) {
  int lo = 0, hi = n - 1;
  const int blk = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bprefix[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  const int ti = order[lo];
  const DevTet &tg = tets[ti];
  // the block's stencil weights in shared memory (reading them from the
  // device array would keep all 100 live in registers)
  __shared__ double sW[kStarPairs];
  __shared__ TR sA[15];
  if (MODE == kOpStar)
    for (int i = threadIdx.x; i < kStarPairs; i += blockDim.x) sW[i] = tg.Wstar[i];
  if (threadIdx.x < 15) sA[threadIdx.x] = (TR)tg.A15[threadIdx.x];
  __syncthreads();
  const int N = tg.N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = ((blk - bprefix[lo]) * 8 + warp) * kResidualCPW;
  TW *r = reinterpret_cast<TW *>(tg.w);
  const StencilData sd{sA, sW, tg.kappa, tg.astore, tg.astride};
  const int *pmap = tg.pk.pw ? tg.pk.row_map : nullptr;
  const TX *xv = xs[ti], *bv = bs[ti];
#pragma unroll 1
  for (int k = 0; k < kResidualCPW && c0 + k < tg.nchunks; ++k) {  // no block-wide synchronisation follows
    const int ch = tg.chunks[c0 + k];
    residual_chunk<TX, TR, TW, MODE>(sd, N, (ch >> 10) & 1023, ch >> 20, 1 + 32 * (ch & 1023), lane, xv, bv, r, pmap,
                                     tg.pk.pw);
  }
}

// ------------------------------------------------- solver vector helpers --
// (full-grid vectors whose boundary entries are zero, except x)

constexpr int kVecBlocks = 512;

template <typename T>
__global__ void __launch_bounds__(256) vec_dot_kernel(const T *__restrict__ a, const T *__restrict__ b, long long n,
                                                      double *__restrict__ partials) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
    acc += (double)a[i] * (double)b[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k];
    partials[blockIdx.x] = s;
  }
}

// y += a x
template <typename T>
__global__ void vec_axpy_kernel(T *__restrict__ y, const T *__restrict__ x, double a, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (T)fma(a, (double)x[i], (double)y[i]);
}

// p = z + b p
template <typename T>
__global__ void vec_xpay_kernel(T *__restrict__ p, const T *__restrict__ z, double b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = (T)fma(b, (double)p[i], (double)z[i]);
}

template <typename TI, typename TO>
__global__ void vec_copy_kernel(TO *__restrict__ dst, const TI *__restrict__ src, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (TO)src[i];
}

// sum of squares of v over the interior points (rows as in the residual)
template <typename T>
__global__ void __launch_bounds__(256) interior_sq_kernel(int N, const T *__restrict__ v, double *__restrict__ partials) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int z = blockIdx.y + 1;
  const int y = blockIdx.x * 8 + warp + 1;
  double acc = 0.0;
  if (y + z <= N - 2) {
    const int64_t r0 = grid_index(N, 0, y, z);
    for (int xx = 1 + lane; xx <= N - 1 - y - z; xx += 32) acc += (double)v[r0 + xx] * (double)v[r0 + xx];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k];
    partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void sum_finish_kernel(const double *__restrict__ partials, int n, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
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

}  // namespace

// ------------------------------------------------------------ launchers --

// 32-point chunks of the interior rows, z-major then y then chunk
int residual_chunks(int N) {
  int n = 0;
  for (int z = 1; z <= N - 3; ++z)
    for (int y = 1; y <= N - 2 - z; ++y) n += (N - 1 - y - z + 31) / 32;
  return n;
}
int residual_blocks(int N) { return (residual_chunks(N) + 8 * kResidualCPW - 1) / (8 * kResidualCPW); }
int rowgrid_blocks(int N) { return ((N - 3 + 7) / 8) * (N - 3); }
void residual_chunk_list(int N, int *out) {
  int i = 0;
  for (int z = 1; z <= N - 3; ++z)
    for (int y = 1; y <= N - 2 - z; ++y)
      for (int c = 0; c < (N - 1 - y - z + 31) / 32; ++c) out[i++] = z << 20 | y << 10 | c;
}

cudaError_t launch_residual(const DevTet &t, int kind, const void *x, const void *b, void *r_out, double *partials,
                            int nblocks_cap, int *nblocks_used, cudaStream_t st, bool packed) {
  if (packed && (!t.pk.pw || kind == kSweepF64)) return cudaErrorInvalidValue;
  const int nb = (t.nchunks + 8 * kResidualCPW - 1) / (8 * kResidualCPW);
  if (nb > nblocks_cap || !t.chunks) return cudaErrorInvalidValue;
  if (nblocks_used) *nblocks_used = nb;
  if (nb == 0) return cudaSuccess;
  dim3 grid(nb);
  const int mode = t.const_kappa ? kOpConst : (t.astore ? kOpStored : kOpStar);
  auto go = [&](auto tx, auto tr, auto tw, auto m) {
    using TX = decltype(tx);
    using TR = decltype(tr);
    using TW = decltype(tw);
    residual_kernel<TX, TR, TW, decltype(m)::value><<<grid, 256, 0, st>>>(t, (const TX *)x, (const TX *)b,
                                                                          (TW *)r_out, partials, packed);
  };
  auto by_mode = [&](auto tx, auto tr, auto tw) {
    if (mode == kOpConst) go(tx, tr, tw, std::integral_constant<int, kOpConst>{});
    else if (mode == kOpStored) go(tx, tr, tw, std::integral_constant<int, kOpStored>{});
    else go(tx, tr, tw, std::integral_constant<int, kOpStar>{});
  };
  if (kind == kSweepF64) by_mode(double{}, double{}, double{});
  else if (kind == kSweepMixed) by_mode(double{}, double{}, float{});
  else by_mode(float{}, float{}, float{});
  return cudaGetLastError();
}

cudaError_t launch_residual_batch(const DevTet *tets, const int *order, const int *bprefix, int n, int total_blocks,
                                  int kind, int op, const void *const *xs, const void *const *bs, cudaStream_t st) {
  if (n <= 0 || total_blocks <= 0) return cudaSuccess;
  auto go = [&](auto tx, auto tr, auto tw, auto m) {
    using TX = decltype(tx);
    using TR = decltype(tr);
    using TW = decltype(tw);
    residual_batch_kernel<TX, TR, TW, decltype(m)::value><<<total_blocks, 256, 0, st>>>(
        tets, order, bprefix, n, reinterpret_cast<const TX *const *>(xs), reinterpret_cast<const TX *const *>(bs));
  };
  auto by_op = [&](auto tx, auto tr, auto tw) {
    if (op == kOpConst) go(tx, tr, tw, std::integral_constant<int, kOpConst>{});
    else if (op == kOpStored) go(tx, tr, tw, std::integral_constant<int, kOpStored>{});
    else go(tx, tr, tw, std::integral_constant<int, kOpStar>{});
  };
  if (kind == kSweepF64) by_op(double{}, double{}, double{});
  else if (kind == kSweepMixed) by_op(double{}, double{}, float{});
  else by_op(float{}, float{}, float{});
  return cudaGetLastError();
}

namespace {
// one warp per 32-point row chunk, as the residual
template <typename TA>
__global__ void __launch_bounds__(256) stencil_store_kernel(DevTet t, TA *__restrict__ A) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ci = blockIdx.x * 8 + warp;
  if (ci >= t.nchunks) return;
  const int ch = t.chunks[ci];
  const int N = t.N, y = (ch >> 10) & 1023, z = ch >> 20, xx = 1 + 32 * (ch & 1023) + lane;
  if (y + z > N - 2 || xx > N - 1 - y - z) return;
  const int64_t r0 = grid_index(N, 0, y, z), rs = grid_index(N, 0, y - 1, z), rn = grid_index(N, 0, y + 1, z);
  const int64_t rb = grid_index(N, 0, y, z - 1), rbn = grid_index(N, 0, y + 1, z - 1);
  const int64_t rt = grid_index(N, 0, y, z + 1), rts = grid_index(N, 0, y - 1, z + 1);
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
  star_store_all(std::make_integer_sequence<int, 15>{}, kq, t.Wstar, A, t.astride, r0 + xx);
}
}  // namespace

cudaError_t launch_stencil_store(const DevTet &t, void *A, bool f32, cudaStream_t st) {
  if (t.const_kappa || !t.kappa || !t.chunks) return cudaErrorInvalidValue;
  const int nb = (t.nchunks + 7) / 8;
  if (nb == 0) return cudaSuccess;
  if (f32)
    stencil_store_kernel<float><<<nb, 256, 0, st>>>(t, static_cast<float *>(A));
  else
    stencil_store_kernel<double><<<nb, 256, 0, st>>>(t, static_cast<double *>(A));
  return cudaGetLastError();
}

template <typename T>
static unsigned vec_blocks(long long n) {
  return (unsigned)std::min<long long>((n + 255) / 256, 4096);
}

cudaError_t launch_dot(bool f64, const void *a, const void *b, long long n, double *partials, double *out,
                       cudaStream_t st) {
  if (f64)
    vec_dot_kernel<double><<<kVecBlocks, 256, 0, st>>>((const double *)a, (const double *)b, n, partials);
  else
    vec_dot_kernel<float><<<kVecBlocks, 256, 0, st>>>((const float *)a, (const float *)b, n, partials);
  sum_finish_kernel<<<1, 256, 0, st>>>(partials, kVecBlocks, out);
  return cudaGetLastError();
}

cudaError_t launch_axpy(bool f64, void *y, const void *x, double a, long long n, cudaStream_t st) {
  if (f64)
    vec_axpy_kernel<double><<<vec_blocks<double>(n), 256, 0, st>>>((double *)y, (const double *)x, a, n);
  else
    vec_axpy_kernel<float><<<vec_blocks<float>(n), 256, 0, st>>>((float *)y, (const float *)x, a, n);
  return cudaGetLastError();
}

cudaError_t launch_xpay(bool f64, void *p, const void *z, double b, long long n, cudaStream_t st) {
  if (f64)
    vec_xpay_kernel<double><<<vec_blocks<double>(n), 256, 0, st>>>((double *)p, (const double *)z, b, n);
  else
    vec_xpay_kernel<float><<<vec_blocks<float>(n), 256, 0, st>>>((float *)p, (const float *)z, b, n);
  return cudaGetLastError();
}

cudaError_t launch_copy(bool src_f64, bool dst_f64, const void *src, void *dst, long long n, cudaStream_t st) {
  const unsigned g = vec_blocks<double>(n);
  if (src_f64 && dst_f64)
    vec_copy_kernel<double, double><<<g, 256, 0, st>>>((double *)dst, (const double *)src, n);
  else if (src_f64)
    vec_copy_kernel<double, float><<<g, 256, 0, st>>>((float *)dst, (const double *)src, n);
  else if (dst_f64)
    vec_copy_kernel<float, double><<<g, 256, 0, st>>>((double *)dst, (const float *)src, n);
  else
    vec_copy_kernel<float, float><<<g, 256, 0, st>>>((float *)dst, (const float *)src, n);
  return cudaGetLastError();
}

cudaError_t launch_interior_norm(int N, bool f64, const void *v, double *partials, int cap, double *out,
                                 cudaStream_t st) {
  dim3 grid((N - 3 + 7) / 8, N - 3);
  if ((int)(grid.x * grid.y) > cap) return cudaErrorInvalidValue;
  if (f64)
    interior_sq_kernel<double><<<grid, 256, 0, st>>>(N, (const double *)v, partials);
  else
    interior_sq_kernel<float><<<grid, 256, 0, st>>>(N, (const float *)v, partials);
  norm_finish_kernel<<<1, 256, 0, st>>>(partials, grid.x * grid.y, out);
  return cudaGetLastError();
}

cudaError_t launch_norm_finish(const double *partials, int n, double *out, cudaStream_t st) {
  norm_finish_kernel<<<1, 256, 0, st>>>(partials, n, out);
  return cudaGetLastError();
}

}  // namespace ilu
