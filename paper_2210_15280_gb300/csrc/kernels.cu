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

// Where a point's operator comes from: the constant stencil (passed in
// registers), or the edge-star weights and kappa at the grid points, or the
// stored coefficients.
struct StencilData {
  const double *Wstar, *kappa;
  const void *astore;  // stored off-diagonal coefficients (MODE 2)
  int64_t astride;
  int plane;           // lanes of the packed array (when r goes there)
};

// MODE of the operator (kernels.cuh): constant stencil, assembled on the fly
// from kappa, or stored coefficients (the same values as on the fly)

// r = b - A x at the interior point of lane `lane` of chunk `ch` (one warp,
// 32 consecutive interior points); returns this lane's share of ||r||^2
// (pmap non-null: r goes to the packed array pw instead, at the slot of the
// point's row, pmap[row id] = forward first step | lane << 20).  A15: the
// constant stencil (registers for FP32, shared memory for FP64).
template <typename TX, typename TR, typename TW, int MODE>
__device__ __forceinline__ double residual_chunk(const StencilData &t, const TR *A15, int N, int ch, int lane,
                                                 const TX *__restrict__ x, const TX *__restrict__ b,
                                                 TW *__restrict__ r, const int *__restrict__ pmap = nullptr,
                                                 float *__restrict__ pw = nullptr) {
  int xx, y, z;
  if (!chunk_point(N, ch, lane, xx, y, z)) return 0.0;
  const StencilRows R = stencil_rows(N, y, z);
  // neighbour values in the order of D: w s se bnw bn bc be c e n nw tse ts tc tw
  TR xv[15];
  xv[0] = (TR)x[R.r0 + xx - 1];
  xv[1] = (TR)x[R.rs + xx];
  xv[2] = (TR)x[R.rs + xx + 1];
  xv[3] = (TR)x[R.rbn + xx - 1];
  xv[4] = (TR)x[R.rbn + xx];
  xv[5] = (TR)x[R.rb + xx];
  xv[6] = (TR)x[R.rb + xx + 1];
  xv[7] = (TR)x[R.r0 + xx];
  xv[8] = (TR)x[R.r0 + xx + 1];
  xv[9] = (TR)x[R.rn + xx];
  xv[10] = (TR)x[R.rn + xx - 1];
  xv[11] = (TR)x[R.rts + xx + 1];
  xv[12] = (TR)x[R.rts + xx];
  xv[13] = (TR)x[R.rt + xx];
  xv[14] = (TR)x[R.rt + xx - 1];
  TR res = (TR)b[R.r0 + xx];
  if (MODE == kOpConst) {
#pragma unroll
    for (int d = 0; d < 15; ++d) res = fma(-A15[d], xv[d], res);
  } else if (MODE == kOpStored) {
    stored_apply(res, t.astore, t.astride, (int64_t)R.r0 + xx, xv);
  } else {
    const double *kap = t.kappa;
    double kq[15];
    kq[0] = kap[R.r0 + xx - 1];
    kq[1] = kap[R.rs + xx];
    kq[2] = kap[R.rs + xx + 1];
    kq[3] = kap[R.rbn + xx - 1];
    kq[4] = kap[R.rbn + xx];
    kq[5] = kap[R.rb + xx];
    kq[6] = kap[R.rb + xx + 1];
    kq[7] = kap[R.r0 + xx];
    kq[8] = kap[R.r0 + xx + 1];
    kq[9] = kap[R.rn + xx];
    kq[10] = kap[R.rn + xx - 1];
    kq[11] = kap[R.rts + xx + 1];
    kq[12] = kap[R.rts + xx];
    kq[13] = kap[R.rt + xx];
    kq[14] = kap[R.rt + xx - 1];
    // the weights are read anew for every point (cached, the same address in
    // every lane): holding all 100 across the chunk loop would take 200 registers
    const double *W = t.Wstar;
    asm volatile("" : "+l"(W));
    star_apply_all(std::make_integer_sequence<int, 15>{}, res, kq, xv, W);
  }
  if (pmap) {
    const int m = pmap[row_id32(N, y, z)];
    pw[packed_index32((m & 0xfffff) + xx - 1, m >> 20, t.plane)] = (float)res;
  } else {
    r[R.r0 + xx] = (TW)res;
  }
  return (double)res * (double)res;
}

// ---- constant stencil: strips.  A warp takes the points (x0 .. x0 + 29, y,
// z) of up to kStripRows consecutive rows y = y0, y0 + 1, ...  Lane l holds
// grid point x0 - 1 + l of every row it loads: lanes 1..30 own the strip's
// points and lanes 0 and 31 only lend their values to the neighbours, which
// take x - 1 and x + 1 from the adjacent lanes.  A point's stencil touches
// the rows (y-1, z) (y, z) (y+1, z) of its layer, (y, z-1) (y+1, z-1) below
// and (y-1, z+1) (y, z+1) above; one row further on, four of them are kept
// and three are loaded (one step ahead, with the next step's b).  The sum
// runs over the directions in the order of the chunk form, so both give the
// same bits.
template <typename TR>
struct StripRow {
  TR m, c, p;  // the row at x - 1, x, x + 1
};
template <typename TR>
__device__ __forceinline__ StripRow<TR> strip_row(TR c) {
  StripRow<TR> r;
  r.c = c;
  r.m = __shfl_up_sync(0xffffffffu, c, 1);
  r.p = __shfl_down_sync(0xffffffffu, c, 1);
  return r;
}
// U: rows unrolled (kStripRows: the rows rotate through registers without
// copies; fewer where the registers do not hold them)
template <typename TX, typename TR, typename TW, int U = kStripRows>
__device__ __forceinline__ double residual_strip(const TR *A15, int N, int strip, int lane,
                                                 const TX *__restrict__ x, const TX *__restrict__ b,
                                                 TW *__restrict__ r, const int *__restrict__ pmap,
                                                 float *__restrict__ pw, int plane) {
  const int x0 = strip & 1023, y0 = (strip >> 10) & 1023, z = strip >> 20;
  const int xl = x0 - 1 + lane;
  const int ny = min(kStripRows, N - z - x0 - y0);  // rows holding a point: x0 + y + z <= N - 1
  // A lane past the end of a row reads a point of a later row instead (the
  // index clamped to the grid's last point): only lanes that own no point of
  // the strip use such a value, so every load is unconditional.
  const int last = (N + 1) * (N + 2) * (N + 3) / 6 - 1;
  auto ld = [&](int i) -> TR { return (TR)x[min(i, last)]; };
  // row y' of layer z' holds x = 0 .. K - y' (K = N - z'): K - y' + 1 points
  const int Kz = N - z, Kb = N - z + 1, Kt = N - z - 1;
  // lane's grid index in the row each layer loads next
  int sz = row_start32(N, y0 - 1, z) + xl, sb = row_start32(N, y0, z - 1) + xl,
      st = row_start32(N, y0 - 1, z + 1) + xl;
  StripRow<TR> zm = strip_row(ld(sz));  // (y0 - 1, z)
  sz += Kz - y0 + 2;
  StripRow<TR> zc = strip_row(ld(sz));  // (y0, z)
  sz += Kz - y0 + 1;
  StripRow<TR> bc = strip_row(ld(sb));  // (y0, z - 1)
  sb += Kb - y0 + 1;
  StripRow<TR> tm = strip_row(ld(st));  // (y0 - 1, z + 1)
  st += Kt - y0 + 2;
  int rc = row_start32(N, y0, z) + xl;
  const int *pm = pmap ? pmap + row_id32(N, y0, z) : nullptr;  // row ids of a layer are consecutive in y
  // the first step's new rows (y0 + 1, z), (y0 + 1, z - 1), (y0, z + 1), its b and packed row
  TR nz = ld(sz), nb = ld(sb), nt = ld(st), nbv = (TR)b[min(rc, last)];
  int npm = pm ? pm[0] : 0;
  double acc2 = 0.0;
#pragma unroll U
  for (int j = 0; j < kStripRows; ++j) {
    if (j >= ny) break;
    const int y = y0 + j;
    const StripRow<TR> zp = strip_row(nz), bp = strip_row(nb), tc = strip_row(nt);
    TR res = nbv;
    const int pmv = npm, rcy = rc;
    // the next step's loads: rows (y + 2, z), (y + 2, z - 1), (y + 1, z + 1)
    sz += Kz - y;
    sb += Kb - y;
    st += Kt - y + 1;
    rc += Kz - y + 1;
    nz = ld(sz);
    nb = ld(sb);
    nt = ld(st);
    nbv = (TR)b[min(rc, last)];
    if (pm && j + 1 < ny) npm = pm[j + 1];
    // w s se bnw bn bc be c e n nw tse ts tc tw
    res = fma(-A15[0], zc.m, res);
    res = fma(-A15[1], zm.c, res);
    res = fma(-A15[2], zm.p, res);
    res = fma(-A15[3], bp.m, res);
    res = fma(-A15[4], bp.c, res);
    res = fma(-A15[5], bc.c, res);
    res = fma(-A15[6], bc.p, res);
    res = fma(-A15[7], zc.c, res);
    res = fma(-A15[8], zc.p, res);
    res = fma(-A15[9], zp.c, res);
    res = fma(-A15[10], zp.m, res);
    res = fma(-A15[11], tm.p, res);
    res = fma(-A15[12], tm.c, res);
    res = fma(-A15[13], tc.c, res);
    res = fma(-A15[14], tc.m, res);
    if (lane >= 1 && lane <= kStripWidth && xl <= N - 1 - y - z) {
      if (pmap)
        pw[packed_index32((pmv & 0xfffff) + xl - 1, pmv >> 20, plane)] = (float)res;
      else
        r[rcy] = (TW)res;
      acc2 += (double)res * (double)res;
    }
    zm = zc;
    zc = zp;
    bc = bp;
    tm = tc;
  }
  return acc2;
}

// CTAs per SM the residual launches are compiled for (their register budget)
// (strips hold seven rows of three values, and the single-tet kernel its
// norm as well: three CTAs, 80 registers, except for the FP32 batch form)
template <int MODE, typename TR, bool BATCH>
constexpr int residual_min_blocks() {
  return MODE == kOpStar ? 2 : (MODE == kOpConst && (sizeof(TR) == 8 || !BATCH) ? 3 : 4);
}

// The constant stencil of a block in the residual type: FP32 coefficients
// stay in registers, FP64 ones (30 registers) are read from shared memory.
template <typename TR, int MODE>
struct ConstStencil {
  TR reg[15];
  __device__ __forceinline__ const TR *load(const double *A, TR *sh) {
    if (MODE != kOpConst) return reg;
    if (sizeof(TR) == 4) {
#pragma unroll
      for (int d = 0; d < 15; ++d) reg[d] = (TR)A[d];
      return reg;
    }
    if (threadIdx.x < 15) sh[threadIdx.x] = (TR)A[threadIdx.x];
    __syncthreads();
    return sh;
  }
};

// One tet: 8 warps per block, warp w of the grid on chunks w, w + W, ... (W
// warps in all; the launch sizes the grid to the CTAs the GPU holds at once,
// so no partial last wave), per-block partial norms.
template <typename TX, typename TR, typename TW, int MODE>
__global__ void __launch_bounds__(256, residual_min_blocks<MODE, TR, false>()) residual_kernel(
    DevTet t, const TX *__restrict__ x, const TX *__restrict__ b, TW *__restrict__ r, double *__restrict__ partials,
    bool packed) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ TR sA15[15];
  ConstStencil<TR, MODE> cs;
  const TR *A15 = cs.load(t.A15, sA15);
  const StencilData sd{t.Wstar, t.kappa, t.astore, t.astride, t.pk.lanes};
  double acc2 = 0.0;
  if constexpr (MODE == kOpConst) {
#pragma unroll 1
    for (int c = blockIdx.x * 8 + warp; c < t.nstrips; c += gridDim.x * 8)  // warp-uniform
      acc2 += residual_strip<TX, TR, TW, sizeof(TR) == 4 ? 4 : 2>(
          A15, t.N, t.strips[c], lane, x, b, r, packed ? t.pk.row_map : nullptr, packed ? t.pk.pw : nullptr,
          t.pk.lanes);
  } else {
#pragma unroll 1
    for (int c = blockIdx.x * 8 + warp; c < t.nchunks; c += gridDim.x * 8)  // warp-uniform
      acc2 += residual_chunk<TX, TR, TW, MODE>(sd, A15, t.N, t.chunks[c], lane, x, b, r,
                                               packed ? t.pk.row_map : nullptr, packed ? t.pk.pw : nullptr);
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

// Many tets whose operators come the same way (MODE): block i belongs to tet
// bmap[i].x and is its block bmap[i].y (laid out as the tet's single-tet
// grid); the result goes to the tet's packed array if it has one, else to
// its scratch w.  One launch per operator kind keeps the register count of
// each kernel that of its own arithmetic.
template <typename TX, typename TR, typename TW, int MODE>
__global__ void __launch_bounds__(256, residual_min_blocks<MODE, TR, true>())
    residual_batch_kernel(const DevTet *__restrict__ tets, const int2 *__restrict__ bmap,
                          const TX *const *__restrict__ xs, const TX *const *__restrict__ bs) {
  const int2 bm = bmap[blockIdx.x];
  const DevTet &tg = tets[bm.x];
  __shared__ TR sA15[15];
  ConstStencil<TR, MODE> cs;
  const TR *A15 = cs.load(tg.A15, sA15);
  const int N = tg.N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = (bm.y * 8 + warp) * kResidualCPW;
  const int nch = tg.nchunks;
  const int *chunks = tg.chunks;
  TW *r = reinterpret_cast<TW *>(tg.w);
  const StencilData sd{tg.Wstar, tg.kappa, tg.astore, tg.astride, tg.pk.lanes};
  const int *pmap = tg.pk.pw ? tg.pk.row_map : nullptr;
  float *pw = tg.pk.pw;
  const TX *xv = xs[bm.x], *bv = bs[bm.x];
  if constexpr (MODE == kOpConst) {  // a strip per warp (no block-wide synchronisation follows)
    const int si = bm.y * 8 + warp;
    if (si < tg.nstrips) residual_strip<TX, TR, TW>(A15, N, tg.strips[si], lane, xv, bv, r, pmap, pw, tg.pk.lanes);
    return;
  }
#pragma unroll 1
  for (int k = 0; k < kResidualCPW && c0 + k < nch; ++k)  // no block-wide synchronisation follows
    residual_chunk<TX, TR, TW, MODE>(sd, A15, N, chunks[c0 + k], lane, xv, bv, r, pmap, pw);
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
int residual_chunks(int N) { return (int)((grid_interior(N) + 31) / 32); }
int residual_blocks(int N) { return (residual_chunks(N) + 8 * kResidualCPW - 1) / (8 * kResidualCPW); }
int rowgrid_blocks(int N) { return ((N - 3 + 7) / 8) * (N - 3); }
void residual_chunk_list(int N, int *out) {
  int i = 0, k = 0;
  for (int z = 1; z <= N - 3; ++z)
    for (int y = 1; y <= N - 2 - z; ++y)
      for (int x = 1; x <= N - 1 - y - z; ++x, ++k)
        if (k % 32 == 0) out[i++] = x | y << 10 | z << 20;
}
// strips: layer z has interior points with x <= N - 2 - z (at y = 1), and
// the strip at x0 rows y with x0 + y + z <= N - 1
template <typename F>
static void for_each_strip(int N, F f) {
  for (int z = 1; z <= N - 3; ++z)
    for (int x0 = 1; x0 <= N - 2 - z; x0 += kStripWidth)
      for (int y0 = 1; x0 + y0 + z <= N - 1; y0 += kStripRows) f(x0 | y0 << 10 | z << 20);
}
int residual_strips(int N) {
  int n = 0;
  for_each_strip(N, [&](int) { ++n; });
  return n;
}
void residual_strip_list(int N, int *out) {
  int i = 0;
  for_each_strip(N, [&](int s) { out[i++] = s; });
}
int residual_strip_blocks(int N) { return (residual_strips(N) + 7) / 8; }

cudaError_t launch_residual(const DevTet &t, int kind, const void *x, const void *b, void *r_out, double *partials,
                            int nblocks_cap, int *nblocks_used, cudaStream_t st, bool packed) {
  if (packed && (!t.pk.pw || kind == kSweepF64)) return cudaErrorInvalidValue;
  if (!t.chunks || !t.strips || nblocks_cap < 1) return cudaErrorInvalidValue;
  const int mode = t.const_kappa ? kOpConst : (t.astore ? kOpStored : kOpStar);
  const int want = ((mode == kOpConst ? t.nstrips : t.nchunks) + 7) / 8;  // a warp per strip or chunk
  if (nblocks_used) *nblocks_used = 0;
  if (want == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  auto go = [&](auto tx, auto tr, auto tw, auto m) {
    using TX = decltype(tx);
    using TR = decltype(tr);
    using TW = decltype(tw);
    auto k = residual_kernel<TX, TR, TW, decltype(m)::value>;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, 0);
    if (e != cudaSuccess) return;
    // as many CTAs as are resident at once (a partial last wave would idle most SMs)
    const int nb = std::max(1, std::min({want, nblocks_cap, std::max(1, per_sm) * sms}));
    if (nblocks_used) *nblocks_used = nb;
    k<<<nb, 256, 0, st>>>(t, (const TX *)x, (const TX *)b, (TW *)r_out, partials, packed);
  };
  auto by_mode = [&](auto tx, auto tr, auto tw) {
    if (mode == kOpConst) go(tx, tr, tw, std::integral_constant<int, kOpConst>{});
    else if (mode == kOpStored) go(tx, tr, tw, std::integral_constant<int, kOpStored>{});
    else go(tx, tr, tw, std::integral_constant<int, kOpStar>{});
  };
  if (kind == kSweepF64) by_mode(double{}, double{}, double{});
  else if (kind == kSweepMixed) by_mode(double{}, double{}, float{});
  else by_mode(float{}, float{}, float{});
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_residual_batch(const DevTet *tets, const int2 *bmap, int total_blocks, int kind, int op,
                                  const void *const *xs, const void *const *bs, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  auto go = [&](auto tx, auto tr, auto tw, auto m) {
    using TX = decltype(tx);
    using TR = decltype(tr);
    using TW = decltype(tw);
    residual_batch_kernel<TX, TR, TW, decltype(m)::value><<<total_blocks, 256, 0, st>>>(
        tets, bmap, reinterpret_cast<const TX *const *>(xs), reinterpret_cast<const TX *const *>(bs));
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
// one warp per 32-point chunk, as the residual
template <typename TA>
__global__ void __launch_bounds__(256) stencil_store_kernel(DevTet t, TA *__restrict__ A) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ci = blockIdx.x * 8 + warp;
  if (ci >= t.nchunks) return;
  const int N = t.N;
  int xx, y, z;
  if (!chunk_point(N, t.chunks[ci], lane, xx, y, z)) return;
  const StencilRows R = stencil_rows(N, y, z);
  const double *kap = t.kappa;
  double kq[15];
  kq[0] = kap[R.r0 + xx - 1];
  kq[1] = kap[R.rs + xx];
  kq[2] = kap[R.rs + xx + 1];
  kq[3] = kap[R.rbn + xx - 1];
  kq[4] = kap[R.rbn + xx];
  kq[5] = kap[R.rb + xx];
  kq[6] = kap[R.rb + xx + 1];
  kq[7] = kap[R.r0 + xx];
  kq[8] = kap[R.r0 + xx + 1];
  kq[9] = kap[R.rn + xx];
  kq[10] = kap[R.rn + xx - 1];
  kq[11] = kap[R.rts + xx + 1];
  kq[12] = kap[R.rts + xx];
  kq[13] = kap[R.rt + xx];
  kq[14] = kap[R.rt + xx - 1];
  star_store_all(std::make_integer_sequence<int, 15>{}, kq, t.Wstar, A, t.astride, (int64_t)R.r0 + xx);
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
