// mg.cu -- geometric multigrid on one macro-tetrahedron (ilu_mg_*).
//
// The hierarchy is the nested family of lattices of levels 2..L of one
// macro-tet (Sec. 2.1): the point c of level l-1 is the point 2c of level l.
// A V-cycle (Sec. 4.2 numerical results) on level l > 2 is
//   nu sweeps of Alg. 2, r = b - A x, b_{l-1} = P^T r, x_{l-1} = 0,
//   V-cycle on level l-1, x += P x_{l-1}, nu sweeps of Alg. 2,
// and on level 2, whose only interior point is (1,1,1), the exact solve
// x = b / A_c.  Sweeps and residuals are those of the level's tet handle.
//
// Grid transfer.  The micro-edges of every level run along the 14
// directions of D (Sec. 2.1), and a fine point F with parity q = F mod 2 != 0
// is the midpoint of exactly one coarse edge: the one along the direction d
// of D with d = q mod 2 (up to sign; the seven classes of q and the seven
// pairs +-d correspond one to one).  So the prolongation of the coarse
// piecewise-linear function is
//   x_F += e(F/2)                          if q = 0,
//   x_F += (e((F-d)/2) + e((F+d)/2)) / 2   otherwise,
// and its transpose, the restriction, is
//   b_c = r(2c) + (1/2) sum_{d in D, d != 0} r(2c + d).
// For an interior coarse point c every 2c + d is an interior fine point, and
// coarse vectors vanish on the boundary, so neither kernel needs a boundary
// test beyond the interior ranges it iterates over.
//
// Both kernels are HBM-bound stencils: a CTA per interior row (y, z), its
// threads along x, so that the reads of each of the (at most nine) rows a
// point touches are coalesced.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "../../include/ilu.h"
#include "hooks.h"
#include "kernels.cuh"

using namespace ilu;

namespace {

ilu_status fail(ilu_status s, const std::string &msg) {
  set_last_error(msg);
  return s;
}

#define MK(call, what)                                                                                  \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return fail(ILU_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define MS(call)                         \
  do {                                   \
    ilu_status s_ = (call);              \
    if (s_ != ILU_OK) return s_;         \
  } while (0)

constexpr int kThreads = 128;

// the representative d in D of the parity class q = (qx, qy, qz) != 0
__device__ __forceinline__ void parity_dir(int qx, int qy, int qz, int &dx, int &dy, int &dz) {
  // e (1,0,0), n (0,1,0), tc (0,0,1), se (1,-1,0), ts (0,-1,1), tw (-1,0,1), tse (1,-1,1)
  dx = qx;
  dy = qy;
  dz = qz;
  if (qx && qy) dy = -1;
  if (qy && qz && !qx) dy = -1;
  if (qx && qz && !qy) dx = -1;
}

// b_c = P^T r_f on the interior of the coarse level (Nc); grid (Nc-3, Nc-3):
// blockIdx.x = y-1, blockIdx.y = z-1
template <typename T>
__global__ void __launch_bounds__(kThreads) restrict_kernel(int Nc, const T *__restrict__ rf, T *__restrict__ bc) {
  const int y = blockIdx.x + 1, z = blockIdx.y + 1;
  if (y + z > Nc - 2) return;
  const int Nf = 2 * Nc;
  const int64_t crow = grid_index(Nc, 0, y, z);
  // fine rows 2y + dy, 2z + dz for dy, dz in {-1, 0, 1}
  int64_t frow[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) frow[a][b] = grid_index(Nf, 0, 2 * y + a - 1, 2 * z + b - 1);
  for (int x = 1 + threadIdx.x; x <= Nc - 1 - y - z; x += kThreads) {
    double half = 0.0;
#pragma unroll
    for (int d = 0; d < kNumDirs; ++d) {
      if (d == kCentre) continue;
      half += (double)rf[frow[dir_dy(d) + 1][dir_dz(d) + 1] + 2 * x + dir_dx(d)];
    }
    bc[crow + x] = (T)((double)rf[frow[1][1] + 2 * x] + 0.5 * half);
  }
}

// x_f += P e_c on the interior of the fine level (Nf); grid (Nf-3, Nf-3)
template <typename T>
__global__ void __launch_bounds__(kThreads) prolong_add_kernel(int Nf, const T *__restrict__ ec, T *__restrict__ xf) {
  const int Y = blockIdx.x + 1, Z = blockIdx.y + 1;
  if (Y + Z > Nf - 2) return;
  const int Nc = Nf / 2;
  const int64_t frow = grid_index(Nf, 0, Y, Z);
  const int qy = Y & 1, qz = Z & 1;
  for (int X = 1 + threadIdx.x; X <= Nf - 1 - Y - Z; X += kThreads) {
    const int qx = X & 1;
    double v;
    if (!(qx | qy | qz)) {
      v = (double)ec[grid_index(Nc, X >> 1, Y >> 1, Z >> 1)];
    } else {
      int dx, dy, dz;
      parity_dir(qx, qy, qz, dx, dy, dz);
      v = 0.5 * ((double)ec[grid_index(Nc, (X - dx) >> 1, (Y - dy) >> 1, (Z - dz) >> 1)] +
                 (double)ec[grid_index(Nc, (X + dx) >> 1, (Y + dy) >> 1, (Z + dz) >> 1)]);
    }
    xf[frow + X] = (T)((double)xf[frow + X] + v);
  }
}

// level 2: x(1,1,1) = b(1,1,1) / A_c (x is zero on entry)
template <typename T>
__global__ void coarse_solve_kernel(const T *__restrict__ b, T *__restrict__ x, double inv_centre) {
  const int64_t i = grid_index(4, 1, 1, 1);
  x[i] = (T)((double)b[i] * inv_centre);
}

template <typename T>
cudaError_t restrict_t(int Nc, const void *rf, void *bc, cudaStream_t st) {
  dim3 grid(Nc - 3, Nc - 3);
  restrict_kernel<T><<<grid, kThreads, 0, st>>>(Nc, (const T *)rf, (T *)bc);
  return cudaGetLastError();
}
template <typename T>
cudaError_t prolong_t(int Nf, const void *ec, void *xf, cudaStream_t st) {
  dim3 grid(Nf - 3, Nf - 3);
  prolong_add_kernel<T><<<grid, kThreads, 0, st>>>(Nf, (const T *)ec, (T *)xf);
  return cudaGetLastError();
}

}  // namespace

struct ilu_mg_s {
  int finest = 0, nu = 0, precision = ILU_MIXED, device = 0;
  bool f64 = true;  // vector type
  double inv_centre = 0.0;
  std::vector<ilu_tet> tets;      // tets[l - 3] smooths level l
  std::vector<void *> x, b, r;    // x[l - 2], b[l - 2]: levels 2..finest-1; r[l - 2]: levels 3..finest
  // Krylov vectors of the finest level and scalars
  void *kr = nullptr, *kz = nullptr, *kp = nullptr, *kq = nullptr, *kzero = nullptr;
  double *d_part = nullptr, *d_scal = nullptr, *h_scal = nullptr;
  int npart = 0;
  bool failed = false;
  size_t elem() const { return f64 ? sizeof(double) : sizeof(float); }
  int N(int l) const { return 1 << l; }
  size_t nodes(int l) const { return (size_t)grid_nodes(1 << l); }
};

namespace {

void free_mg(ilu_mg m) {
  for (ilu_tet t : m->tets) ilu_destroy(t);
  if (m->device >= 0) cudaSetDevice(m->device);
  for (auto *v : {&m->x, &m->b, &m->r})
    for (void *p : *v) cudaFree(p);
  for (void *p : {m->kr, m->kz, m->kp, m->kq, m->kzero}) cudaFree(p);
  cudaFree(m->d_part);
  cudaFree(m->d_scal);
  cudaFreeHost(m->h_scal);
}

ilu_status restrict_to(ilu_mg m, int l, cudaStream_t st) {  // r[l] -> b[l-1]
  const int Nc = m->N(l - 1);
  MK(m->f64 ? restrict_t<double>(Nc, m->r[l - 2], m->b[l - 3], st) : restrict_t<float>(Nc, m->r[l - 2], m->b[l - 3], st),
     "restriction launch");
  return ILU_OK;
}

// one V-cycle on level l for vectors x, b of that level
ilu_status vcycle(ilu_mg m, int l, void *x, const void *b, cudaStream_t st) {
  if (l == 2) {
    if (m->f64)
      coarse_solve_kernel<double><<<1, 1, 0, st>>>((const double *)b, (double *)x, m->inv_centre);
    else
      coarse_solve_kernel<float><<<1, 1, 0, st>>>((const float *)b, (float *)x, m->inv_centre);
    MK(cudaGetLastError(), "coarse solve launch");
    return ILU_OK;
  }
  ilu_tet t = m->tets[l - 3];
  MS(tet_sweeps(t, x, b, m->nu, st));
  MS(tet_residual(t, x, b, m->r[l - 2], nullptr, st));
  MS(restrict_to(m, l, st));
  void *xc = m->x[l - 3];
  MK(cudaMemsetAsync(xc, 0, m->nodes(l - 1) * m->elem(), st), "clear coarse x");
  MS(vcycle(m, l - 1, xc, m->b[l - 3], st));
  MK(m->f64 ? prolong_t<double>(m->N(l), xc, x, st) : prolong_t<float>(m->N(l), xc, x, st), "prolongation launch");
  MS(tet_sweeps(t, x, b, m->nu, st));
  return ILU_OK;
}

ilu_status check_mg(ilu_mg m) {
  if (!m) return fail(ILU_EINVAL, "null multigrid handle");
  if (m->failed) return fail(ILU_ECUDA, "multigrid handle failed earlier; destroy it");
  return ILU_OK;
}

ilu_status read_scalar(ilu_mg m, int n, cudaStream_t st) {
  MK(cudaMemcpyAsync(m->h_scal, m->d_scal, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "scalar copy");
  return tet_check(m->tets.back(), st);  // synchronises; reports timed-out waits
}

// ||v|| over the finest interior into h_scal[slot]
ilu_status finest_norm(ilu_mg m, const void *v, int slot, cudaStream_t st) {
  MK(launch_interior_norm(m->N(m->finest), m->f64, v, m->d_part, m->npart, m->d_scal + slot, st), "norm launch");
  return ILU_OK;
}

ilu_status fail_mg(ilu_mg m, ilu_status s) {
  m->failed = true;
  return s;
}

}  // namespace

extern "C" {

ilu_status ilu_mg_setup(const double macro_tet[12], int level, const ilu_coeff *coeff, int poly_degree, int nu,
                        const ilu_opts *opts, ilu_mg *out) {
  ilu::DeviceRestore keep_device;
  if (!out) return fail(ILU_EINVAL, "null output handle");
  *out = nullptr;
  if (level < 3 || level > 10) return fail(ILU_EINVAL, "multigrid level out of [3, 10]");
  if (nu < 1 || nu > 16) return fail(ILU_EINVAL, "smoothing steps out of [1, 16]");
  ilu_opts o;
  ilu_opts_default(&o);
  if (opts) o = *opts;
  if (o.device < 0) return fail(ILU_ENODEV, "multigrid needs a device");
  ilu_mg m = new (std::nothrow) ilu_mg_s;
  if (!m) return fail(ILU_ENOMEM, "out of host memory");
  m->finest = level;
  m->nu = nu;
  m->precision = o.precision;
  m->device = o.device;
  m->f64 = o.precision != ILU_F32;
  auto bail = [&](ilu_status s) {
    free_mg(m);
    delete m;
    return s;
  };
  // level 2: the stencil centre at its one interior point, from a host-only set-up
  {
    ilu_opts ho = o;
    ho.device = -1;
    ilu_tet h = nullptr;
    ilu_status s = ilu_setup(macro_tet, 2, coeff, poly_degree, &ho, &h);
    if (s != ILU_OK) return bail(s);
    double st15[15];
    s = ilu_stencil(h, 1, 1, 1, st15);
    ilu_destroy(h);
    if (s != ILU_OK) return bail(s);
    if (!(st15[kCentre] > 0.0)) return bail(fail(ILU_ESINGULAR, "non-positive coarse diagonal"));
    m->inv_centre = 1.0 / st15[kCentre];
  }
  for (int l = 3; l <= level; ++l) {
    ilu_tet t = nullptr;
    ilu_status s = ilu_setup(macro_tet, l, coeff, poly_degree, &o, &t);
    if (s != ILU_OK) return bail(s);
    m->tets.push_back(t);
  }
  if (cudaSetDevice(m->device) != cudaSuccess) return bail(fail(ILU_ECUDA, "cudaSetDevice"));
  auto alloc = [&](void **p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) return false;
    return cudaMemset(*p, 0, bytes) == cudaSuccess;
  };
  m->x.assign(level - 1, nullptr);
  m->b.assign(level - 1, nullptr);
  m->r.assign(level - 1, nullptr);
  for (int l = 2; l <= level; ++l) {
    const size_t bytes = m->nodes(l) * m->elem();
    if (l < level && (!alloc(&m->x[l - 2], bytes) || !alloc(&m->b[l - 2], bytes)))
      return bail(fail(ILU_ENOMEM, "cudaMalloc level vectors"));
    if (l >= 3 && !alloc(&m->r[l - 2], bytes)) return bail(fail(ILU_ENOMEM, "cudaMalloc level residual"));
  }
  const size_t fb = m->nodes(level) * m->elem();
  for (void **p : {&m->kr, &m->kz, &m->kp, &m->kq, &m->kzero})
    if (!alloc(p, fb)) return bail(fail(ILU_ENOMEM, "cudaMalloc Krylov vectors"));
  m->npart = std::max(kDotPartials, rowgrid_blocks(m->N(level)));
  if (cudaMalloc(&m->d_part, sizeof(double) * m->npart) != cudaSuccess ||
      cudaMalloc(&m->d_scal, sizeof(double) * 8) != cudaSuccess ||
      cudaMallocHost(&m->h_scal, sizeof(double) * 8) != cudaSuccess)
    return bail(fail(ILU_ENOMEM, "cudaMalloc scalars"));
  *out = m;
  return ILU_OK;
}

ilu_status ilu_mg_destroy(ilu_mg m) {
  ilu::DeviceRestore keep_device;
  if (!m) return ILU_OK;
  free_mg(m);
  delete m;
  return ILU_OK;
}

ilu_status ilu_mg_level(ilu_mg m, int level, ilu_tet *out) {
  if (!m || !out) return fail(ILU_EINVAL, "null argument");
  if (level < 3 || level > m->finest) return fail(ILU_EINVAL, "level out of the hierarchy's smoothed levels");
  *out = m->tets[level - 3];
  return ILU_OK;
}

ilu_status ilu_mg_cycle(ilu_mg m, void *x, const void *b, int cycles, void *stream, double *res_norms) {
  ilu::DeviceRestore keep_device;
  MS(check_mg(m));
  if (!x || !b) return fail(ILU_EINVAL, "null vector");
  if (cycles < 0) return fail(ILU_EINVAL, "negative cycle count");
  cudaStream_t st = (cudaStream_t)stream;
  MK(cudaSetDevice(m->device), "cudaSetDevice");
  ilu_tet tf = m->tets.back();
  for (int k = 0; k < cycles; ++k) {
    ilu_status s = vcycle(m, m->finest, x, b, st);
    if (s != ILU_OK) return fail_mg(m, s);
    if (res_norms) {
      s = tet_residual(tf, x, b, m->kr, m->d_scal, st);
      if (s == ILU_OK) s = read_scalar(m, 1, st);
      if (s != ILU_OK) return fail_mg(m, s);
      res_norms[k] = m->h_scal[0];
    }
  }
  return ILU_OK;
}

ilu_status ilu_mg_solve(ilu_mg m, void *x, const void *b, int method, double rtol, int max_iter, void *stream,
                        int *iters, double *rel_res) {
  ilu::DeviceRestore keep_device;
  MS(check_mg(m));
  if (!x || !b) return fail(ILU_EINVAL, "null vector");
  if (method == ILU_MG_VCYCLE) method = ILU_RICHARDSON;
  if (method == ILU_MG_PCG) method = ILU_PCG;
  if (method != ILU_RICHARDSON && method != ILU_PCG) return fail(ILU_EINVAL, "unknown method");
  if (!(rtol >= 0.0) || max_iter < 0) return fail(ILU_EINVAL, "bad tolerance or iteration limit");
  cudaStream_t st = (cudaStream_t)stream;
  MK(cudaSetDevice(m->device), "cudaSetDevice");
  ilu_tet tf = m->tets.back();
  const long long n = (long long)m->nodes(m->finest);
  const bool f64 = m->f64;
  if (iters) *iters = 0;
  if (rel_res) *rel_res = 0.0;
  MS(finest_norm(m, b, 0, st));
  MS(read_scalar(m, 1, st));
  double bn = m->h_scal[0];
  if (bn == 0.0) bn = 1.0;
  ilu_status s;
  auto resid = [&](double &rel) -> ilu_status {  // kr = b - A x, rel = ||kr|| / ||b||
    MS(tet_residual(tf, x, b, m->kr, m->d_scal, st));
    MS(read_scalar(m, 1, st));
    rel = m->h_scal[0] / bn;
    return ILU_OK;
  };
  double rel = 0.0;
  if (method == ILU_RICHARDSON) {
    for (int it = 0;; ++it) {
      if ((s = resid(rel)) != ILU_OK) return fail_mg(m, s);
      if (iters) *iters = it;
      if (rel_res) *rel_res = rel;
      if (rel <= rtol) return ILU_OK;
      if (it == max_iter) return fail(ILU_ENOTCONV, "V-cycle iteration reached max_iter");
      if ((s = vcycle(m, m->finest, x, b, st)) != ILU_OK) return fail_mg(m, s);
    }
  }
  // CG preconditioned by one V-cycle from zero
  if ((s = resid(rel)) != ILU_OK) return fail_mg(m, s);
  double rz_old = 0.0;
  for (int it = 0;; ++it) {
    if (iters) *iters = it;
    if (rel_res) *rel_res = rel;
    if (rel <= rtol) return ILU_OK;
    if (it == max_iter) return fail(ILU_ENOTCONV, "multigrid-preconditioned CG reached max_iter");
    MK(cudaMemsetAsync(m->kz, 0, n * m->elem(), st), "clear z");
    if ((s = vcycle(m, m->finest, m->kz, m->kr, st)) != ILU_OK) return fail_mg(m, s);
    MK(launch_dot(f64, m->kr, m->kz, n, m->d_part, m->d_scal, st), "dot launch");
    if ((s = read_scalar(m, 1, st)) != ILU_OK) return fail_mg(m, s);
    const double rz = m->h_scal[0];
    if (it == 0)
      MK(launch_copy(f64, f64, m->kz, m->kp, n, st), "copy launch");
    else
      MK(launch_xpay(f64, m->kp, m->kz, rz / rz_old, n, st), "xpay launch");
    rz_old = rz;
    // q = -A p (residual with b = 0; p vanishes on the boundary)
    if ((s = tet_residual(tf, m->kp, m->kzero, m->kq, nullptr, st)) != ILU_OK) return fail_mg(m, s);
    MK(launch_dot(f64, m->kp, m->kq, n, m->d_part, m->d_scal, st), "dot launch");
    if ((s = read_scalar(m, 1, st)) != ILU_OK) return fail_mg(m, s);
    const double pAp = -m->h_scal[0];
    if (!(pAp > 0.0)) return fail(ILU_ESINGULAR, "CG met a non-positive curvature");
    const double alpha = rz / pAp;
    MK(launch_axpy(f64, x, m->kp, alpha, n, st), "axpy launch");
    MK(launch_axpy(f64, m->kr, m->kq, alpha, n, st), "axpy launch");
    MK(launch_dot(f64, m->kr, m->kr, n, m->d_part, m->d_scal, st), "dot launch");
    if ((s = read_scalar(m, 1, st)) != ILU_OK) return fail_mg(m, s);
    rel = std::sqrt(std::max(m->h_scal[0], 0.0)) / bn;
  }
}

ilu_status ilu_mg_rate(ilu_mg m, void *e, int steps, void *stream, double *rho, double *history) {
  ilu::DeviceRestore keep_device;
  MS(check_mg(m));
  if (!e || !rho) return fail(ILU_EINVAL, "null argument");
  if (steps < 1) return fail(ILU_EINVAL, "steps must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  MK(cudaSetDevice(m->device), "cudaSetDevice");
  const long long n = (long long)m->nodes(m->finest);
  ilu_status s;
  MS(finest_norm(m, e, 0, st));
  if ((s = read_scalar(m, 1, st)) != ILU_OK) return fail_mg(m, s);
  if (!(m->h_scal[0] > 0.0)) return fail(ILU_EINVAL, "zero start error");
  double scale = 1.0 / m->h_scal[0];
  for (int k = 0; k < steps; ++k) {
    MK(launch_xpay(m->f64, e, m->kzero, scale, n, st), "scale launch");  // e = 0 + scale e
    if ((s = vcycle(m, m->finest, e, m->kzero, st)) != ILU_OK) return fail_mg(m, s);
    MS(finest_norm(m, e, 0, st));
    if ((s = read_scalar(m, 1, st)) != ILU_OK) return fail_mg(m, s);
    const double r = m->h_scal[0];
    if (history) history[k] = r;
    *rho = r;
    if (!(r > 0.0)) break;  // exact solve: the error vanished
    scale = 1.0 / r;
  }
  return ILU_OK;
}

}  // extern "C"
