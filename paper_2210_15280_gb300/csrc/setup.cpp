// setup.cpp -- FP64 host set-up of one macro-tetrahedron (arXiv 2210.15280,
// Sec. 2.1, Sec. 3 and Sec. 4.1):
//   * affine map of the logical grid and the six classes of micro-tetrahedra,
//   * the operator stencil A^p_d (constant coefficient: 15 numbers; variable
//     coefficient: edge-star weights applied to kappa at the grid points),
//   * the streaming ILU(0) factorisation of the interior block, solved from
//     the general stencil equation  A^p_d = sum_e L^p_e D^{p+e} L^{p+d}_{e-d}
//     (Sec. 3) with O(N^2) storage (two face layers, as in Alg. 1),
//   * the sample sets S_d and the ridge-regularised least-squares fit of the
//     eight surrogates in the tensor space P_{dgx,dgy,dgz} (Sec. 4.1),
//   * the per-row evaluation tables used by the sweep kernels: each surrogate
//     restricted to an interior row (y,z) is a polynomial of degree dgx in
//     t = h (x - xc), xc the row centre; the backward table holds 1/D and the
//     L_d shifted to p - d, so that the backward sweep evaluates L^{p-d}_d at p.
#include "setup.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>

namespace ilu {

namespace {

int dir_of(int ox, int oy, int oz) {
  for (int d = 0; d < kNumDirs; ++d)
    if (dir_dx(d) == ox && dir_dy(d) == oy && dir_dz(d) == oz) return d;
  return -1;
}

void legendre_all(int n, double u, double *p) {
  p[0] = 1.0;
  if (n >= 1) p[1] = u;
  for (int k = 1; k < n; ++k) p[k + 1] = ((2 * k + 1) * u * p[k] - k * p[k - 1]) / (k + 1);
}

// Monomial coefficients (in t) of P_0..P_n evaluated at 2t + a.
// out[i*(n+1) + k] = coefficient of t^k in P_i(2t + a).
void legendre_shifted_monomials(int n, double a, double *out) {
  const int S = n + 1;
  std::fill(out, out + S * S, 0.0);
  out[0] = 1.0;
  if (n >= 1) { out[S + 0] = a; out[S + 1] = 2.0; }
  for (int i = 1; i < n; ++i) {
    double *pn = out + i * S, *pm = out + (i - 1) * S, *pq = out + (i + 1) * S;
    for (int k = 0; k <= n; ++k) {
      double v = (2 * i + 1) * a * pn[k] - i * pm[k];
      if (k > 0) v += (2 * i + 1) * 2.0 * pn[k - 1];
      pq[k] = v / (i + 1);
    }
  }
}

// Householder QR least squares: minimise ||A c - t|| for a column-major
// m x n matrix with m >= n; A and t are overwritten.  Returns false on a
// zero column.
bool householder_lsq(int m, int n, std::vector<double> &A, std::vector<double> &t, double *c) {
  std::vector<double> beta(n);
  for (int k = 0; k < n; ++k) {
    double *ak = &A[(size_t)k * m];
    double s = 0.0;
    for (int i = k; i < m; ++i) s += ak[i] * ak[i];
    double nrm = std::sqrt(s);
    if (nrm == 0.0) return false;
    double alpha = ak[k] > 0 ? -nrm : nrm;
    double v0 = ak[k] - alpha;
    // v = (v0, ak[k+1..m-1]); H = I - 2 v v^T / (v^T v)
    double vtv = v0 * v0 + (s - ak[k] * ak[k]);
    ak[k] = v0;
    beta[k] = vtv > 0 ? 2.0 / vtv : 0.0;
    for (int j = k + 1; j < n; ++j) {
      double *aj = &A[(size_t)j * m];
      double w = 0.0;
      for (int i = k; i < m; ++i) w += ak[i] * aj[i];
      w *= beta[k];
      for (int i = k; i < m; ++i) aj[i] -= w * ak[i];
    }
    double w = 0.0;
    for (int i = k; i < m; ++i) w += ak[i] * t[i];
    w *= beta[k];
    for (int i = k; i < m; ++i) t[i] -= w * ak[i];
    ak[k] = alpha;  // R diagonal; the Householder vector's head is no longer needed
  }
  for (int k = n - 1; k >= 0; --k) {
    double v = t[k];
    for (int j = k + 1; j < n; ++j) v -= A[(size_t)j * m + k] * c[j];
    c[k] = v / A[(size_t)k * m + k];
  }
  return true;
}

}  // namespace

void host_phys(const HostTet &t, double x, double y, double z, double X[3]) {
  for (int c = 0; c < 3; ++c)
    X[c] = t.P[0][c] + ((t.P[1][c] - t.P[0][c]) * x + (t.P[2][c] - t.P[0][c]) * y + (t.P[3][c] - t.P[0][c]) * z) / t.N;
}

double host_kappa(const ilu_coeff &c, const double X[3]) {
  switch (c.kind) {
    case ILU_COEFF_CONST: return c.c0;
    case ILU_COEFF_SINPROD:
      return c.c0 + c.amp * std::sin(2.0 * M_PI * X[0]) * std::sin(2.0 * M_PI * X[1]) * std::sin(2.0 * M_PI * X[2]);
    default:
      return 1.0 + 10.0 * (std::pow(X[0], c.ipow) + std::pow(X[1], c.ipow) + std::pow(X[2], c.ipow));
  }
}

// Six classes of micro-tetrahedra: images of the Kuhn simplices of the lattice
// basis a = e, b = ts, c = bc, i.e. {0, s0, s0+s1, a+b+c} for the six orders
// (s0, s1, s2) of (a, b, c).  Their unit-coefficient element matrices
// |T| grad(phi_i).grad(phi_j) are the same for every tetrahedron of a class
// because the map to physical space is affine.
static void element_classes(HostTet &t) {
  const int basis[3][3] = {{1, 0, 0}, {0, -1, 1}, {0, 0, -1}};
  const int order[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
  for (int cl = 0; cl < 6; ++cl) {
    for (int c = 0; c < 3; ++c) {
      t.off[cl][0][c] = 0;
      t.off[cl][1][c] = basis[order[cl][0]][c];
      t.off[cl][2][c] = basis[order[cl][0]][c] + basis[order[cl][1]][c];
      t.off[cl][3][c] = basis[0][c] + basis[1][c] + basis[2][c];
    }
    double E[3][3];  // E[m] = physical edge vector from vertex 0 to vertex m+1
    for (int m = 0; m < 3; ++m) {
      double X0[3], X1[3];
      host_phys(t, 0, 0, 0, X0);
      host_phys(t, t.off[cl][m + 1][0], t.off[cl][m + 1][1], t.off[cl][m + 1][2], X1);
      for (int c = 0; c < 3; ++c) E[m][c] = X1[c] - X0[c];
    }
    auto cross = [](const double *u, const double *v, double *w) {
      w[0] = u[1] * v[2] - u[2] * v[1];
      w[1] = u[2] * v[0] - u[0] * v[2];
      w[2] = u[0] * v[1] - u[1] * v[0];
    };
    double g[4][3], c23[3], c31[3], c12[3];
    cross(E[1], E[2], c23);
    cross(E[2], E[0], c31);
    cross(E[0], E[1], c12);
    double det = E[0][0] * c23[0] + E[0][1] * c23[1] + E[0][2] * c23[2];
    for (int c = 0; c < 3; ++c) {
      g[1][c] = c23[c] / det;
      g[2][c] = c31[c] / det;
      g[3][c] = c12[c] / det;
      g[0][c] = -(g[1][c] + g[2][c] + g[3][c]);
    }
    double vol = std::fabs(det) / 6.0;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        t.Kunit[cl][i][j] = vol * (g[i][0] * g[j][0] + g[i][1] * g[j][1] + g[i][2] * g[j][2]);
  }
}

// Constant stencil (unit coefficient) and edge-star weights: loop over the 24
// micro-tetrahedra around an interior point (class cl, local position loc).
static bool stencil_weights(HostTet &t, std::string &err) {
  double A1[15] = {};
  std::memset(t.W, 0, sizeof(t.W));
  for (int cl = 0; cl < 6; ++cl)
    for (int loc = 0; loc < 4; ++loc) {
      int rel[4];
      for (int m = 0; m < 4; ++m) {
        rel[m] = dir_of(t.off[cl][m][0] - t.off[cl][loc][0], t.off[cl][m][1] - t.off[cl][loc][1],
                        t.off[cl][m][2] - t.off[cl][loc][2]);
        if (rel[m] < 0) { err = "micro-tetrahedron edge outside the stencil set"; return false; }
      }
      for (int j = 0; j < 4; ++j) {
        A1[rel[j]] += t.Kunit[cl][loc][j];
        if (j == loc) continue;
        for (int m = 0; m < 4; ++m) t.W[rel[j]][rel[m]] += 0.25 * t.Kunit[cl][loc][j];
      }
    }
  for (int d = 0; d < 15; ++d) t.A15[d] = (t.coeff.kind == ILU_COEFF_CONST ? t.coeff.c0 : 1.0) * A1[d];
  // every nonzero weight must lie on the fixed pattern the kernels unroll
  bool on[15][15] = {};
  for (int e = 0; e < kStarPairs; ++e) {
    on[star_d(e)][star_q(e)] = true;
    t.Wstar[e] = t.W[star_d(e)][star_q(e)];
  }
  for (int d = 0; d < 15; ++d)
    for (int q = 0; q < 15; ++q)
      if (t.W[d][q] != 0.0 && !on[d][q]) { err = "edge-star weight off the fixed pattern"; return false; }
  return true;
}

bool unit_stencil(const double P[12], double A[15], std::string &err) {
  double e[3][3], scale = 0.0;
  for (int k = 0; k < 12; ++k)
    if (!std::isfinite(P[k])) { err = "macro-tetrahedron has non-finite coordinates"; return false; }
  for (int m = 0; m < 3; ++m)
    for (int c = 0; c < 3; ++c) {
      e[m][c] = P[3 * (m + 1) + c] - P[c];
      scale = std::max(scale, std::fabs(e[m][c]));
    }
  const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                     e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
  if (!(std::fabs(det) > 1e-12 * scale * scale * scale)) { err = "degenerate macro-tetrahedron"; return false; }
  HostTet t;
  t.L = 2;
  t.N = 4;
  t.h = 0.25;
  std::memcpy(t.P, P, sizeof(double) * 12);
  t.coeff = ilu_coeff{ILU_COEFF_CONST, 1.0, 0.0, 0};
  t.const_kappa = true;
  element_classes(t);
  if (!stencil_weights(t, err)) return false;
  std::memcpy(A, t.A15, sizeof(double) * 15);
  return true;
}

void host_stencil(const HostTet &t, int x, int y, int z, double A[15]) {
  if (t.const_kappa) {
    for (int d = 0; d < 15; ++d) A[d] = t.A15[d];
    return;
  }
  double kq[15];
  for (int q = 0; q < 15; ++q) {
    int qx = x + dir_dx(q), qy = y + dir_dy(q), qz = z + dir_dz(q);
    kq[q] = in_grid(t.N, qx, qy, qz) ? t.kappa[grid_index(t.N, qx, qy, qz)] : 0.0;
  }
  double sum = 0.0;
  for (int d = 0; d < 15; ++d) {
    if (d == kCentre) continue;
    double a = 0.0;
    for (int q = 0; q < 15; ++q) a += t.W[d][q] * kq[q];
    A[d] = a;
    sum += a;
  }
  A[kCentre] = -sum;  // rows of the stiffness matrix sum to zero
}

double host_eval_coefs(const HostTet &t, int f, double x, double y, double z) {
  double px[16], py[16], pz[16];
  legendre_all(t.deg[0], 2 * t.h * x - 1, px);
  legendre_all(t.deg[1], 2 * t.h * y - 1, py);
  legendre_all(t.deg[2], 2 * t.h * z - 1, pz);
  const double *c = &t.coefs[(size_t)f * t.M];
  double s = 0.0;
  for (int i = 0; i <= t.deg[0]; ++i)
    for (int j = 0; j <= t.deg[1]; ++j)
      for (int k = 0; k <= t.deg[2]; ++k) s += c[(i * (t.deg[1] + 1) + j) * (t.deg[2] + 1) + k] * px[i] * py[j] * pz[k];
  return s;
}

// The row polynomial in t = h (x - xc) of surrogate f evaluated at
// (x + sx, y + sy, z + sz) for x on row (y, z).
static void row_poly(const HostTet &t, int f, int y, int z, int sx, int sy, int sz, double *out) {
  const int n = t.deg[0];
  double py[16], pz[16], q[16], mono[17 * 17];
  legendre_all(t.deg[1], 2 * t.h * (y + sy) - 1, py);
  legendre_all(t.deg[2], 2 * t.h * (z + sz) - 1, pz);
  const double *c = &t.coefs[(size_t)f * t.M];
  for (int i = 0; i <= n; ++i) {
    double s = 0.0;
    for (int j = 0; j <= t.deg[1]; ++j)
      for (int k = 0; k <= t.deg[2]; ++k) s += c[(i * (t.deg[1] + 1) + j) * (t.deg[2] + 1) + k] * py[j] * pz[k];
    q[i] = s;
  }
  // u_x = 2 h (x + sx) - 1 = 2 t + a with x = xc + t/h
  const double xc = 0.5 * (t.N - y - z);
  const double a = 2 * t.h * (xc + sx) - 1;
  legendre_shifted_monomials(n, a, mono);
  for (int k = 0; k <= n; ++k) {
    double s = 0.0;
    for (int i = 0; i <= n; ++i) s += q[i] * mono[i * (n + 1) + k];
    out[k] = s;
  }
}

void build_row_tables(HostTet &t) {
  const int N = t.N;
  const int64_t R = num_rows(N);
  t.dx = t.deg[0];
  // coefficients per function, zero padded to 4, 8 or 16 so that a row block
  // is a whole number of 16-byte chunks and Horner can run over the padding
  t.rstride = t.dx + 1 <= 4 ? 4 : (t.dx + 1 <= 8 ? 8 : 16);
  const int S = t.rstride;
  t.tabF64.assign((size_t)R * 7 * S, 0.0);
  t.tabB64.assign((size_t)R * 8 * S, 0.0);
  auto work = [&](int z0, int z1) {
    for (int z = z0; z < z1; ++z)
      for (int y = 1; y <= N - 2 - z; ++y) {
        const int64_t r = row_id(N, y, z);
        for (int d = 0; d < kNumLower; ++d) row_poly(t, d, y, z, 0, 0, 0, &t.tabF64[((size_t)r * 7 + d) * S]);
        row_poly(t, 7, y, z, 0, 0, 0, &t.tabB64[((size_t)r * 8 + 0) * S]);
        for (int d = 0; d < kNumLower; ++d)
          row_poly(t, d, y, z, -dir_dx(d), -dir_dy(d), -dir_dz(d), &t.tabB64[((size_t)r * 8 + 1 + d) * S]);
      }
  };
  const int nth = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  const int zmax = N - 3;
  for (int k = 0; k < nth; ++k) {
    int a = 1 + (int)((int64_t)zmax * k / nth), b = 1 + (int)((int64_t)zmax * (k + 1) / nth);
    if (a < b) pool.emplace_back(work, a, b);
  }
  for (auto &th : pool) th.join();
  // FP32 tables: four function pairs per row, coefficient k of functions
  // (2p, 2p+1) side by side, so that the sweep evaluates two polynomials per
  // packed FMA; the forward table gets a zero eighth function
  t.tabF32.assign((size_t)R * 8 * S, 0.0f);
  t.tabB32.assign((size_t)R * 8 * S, 0.0f);
  for (int64_t r = 0; r < R; ++r)
    for (int f = 0; f < 8; ++f)
      for (int k = 0; k < S; ++k) {
        const size_t o = (((size_t)r * 4 + f / 2) * S + k) * 2 + (f & 1);
        if (f < 7) t.tabF32[o] = (float)t.tabF64[((size_t)r * 7 + f) * S + k];
        t.tabB32[o] = (float)t.tabB64[((size_t)r * 8 + f) * S + k];
      }
}

static double horner(const double *c, int n, double tt) {
  double v = c[n];
  for (int k = n - 1; k >= 0; --k) v = v * tt + c[k];
  return v;
}

void host_eval_tables(const HostTet &t, int x, int y, int z, double out[8]) {
  const int N = t.N;
  const int64_t r = row_id(N, y, z);
  const double tt = t.h * (x - 0.5 * (N - y - z));
  for (int d = 0; d < kNumLower; ++d)
    out[d] = in_interior(N, x + dir_dx(d), y + dir_dy(d), z + dir_dz(d))
                 ? horner(&t.tabF64[((size_t)r * 7 + d) * t.rstride], t.dx, tt)
                 : 0.0;
  out[7] = horner(&t.tabB64[((size_t)r * 8) * t.rstride], t.dx, tt);
}

namespace {

// Order of the unknowns at a point and the terms of each stencil equation
// A^p_d = L^p_d D^{p+d} + sum_{e != d, e - d in D_l} L^p_e D^{p+e} L^{p+d}_{e-d}.
struct FactorPlan {
  int order[7];
  int nterm[7];
  int e[7][7], f[7][7];  // term k of unknown d: e = d~, f = index of (e - d) in D_l
};

FactorPlan make_plan() {
  FactorPlan pl = {};
  bool dep[7][7] = {};
  for (int d = 0; d < 7; ++d) {
    pl.nterm[d] = 0;
    for (int e = 0; e < 7; ++e) {
      if (e == d) continue;
      int fd = dir_of(dir_dx(e) - dir_dx(d), dir_dy(e) - dir_dy(d), dir_dz(e) - dir_dz(d));
      if (fd >= 0 && fd < 7) {
        pl.e[d][pl.nterm[d]] = e;
        pl.f[d][pl.nterm[d]] = fd;
        pl.nterm[d]++;
        dep[d][e] = true;
      }
    }
  }
  bool done[7] = {};
  int k = 0;
  while (k < 7) {
    for (int d = 0; d < 7; ++d) {
      if (done[d]) continue;
      bool ready = true;
      for (int e = 0; e < 7; ++e)
        if (dep[d][e] && !done[e]) ready = false;
      if (ready) { pl.order[k++] = d; done[d] = true; }
    }
  }
  return pl;
}

struct Sample {
  int x, y, z;
  double v;
};

}  // namespace

// Streaming factorisation + samples.  Layer buffers hold, for every (x, y) of
// the current and the previous face layer, the 7 factor entries and the pivot
// (defaults L = 0, D = 1 off the interior, as Alg. 1 initialises them).
// The recursion is sequential in lexicographic order.  The operator stencils
// it consumes are not: for a variable coefficient, worker threads assemble
// the stencils of face layer z + 1 while this thread factors layer z.
static ilu_status factorise(HostTet &t, std::vector<Sample> samples[8], std::string &err) {
  const int N = t.N;
  const int S = N + 2;
  const FactorPlan pl = make_plan();
  std::vector<double> lay[2];
  for (int k = 0; k < 2; ++k) lay[k].assign((size_t)S * S * 8, 0.0);
  auto reset = [&](std::vector<double> &b) {
    for (size_t i = 0; i < b.size(); i += 8) {
      std::fill(&b[i], &b[i] + 7, 0.0);
      b[i + 7] = 1.0;
    }
  };
  reset(lay[0]);
  reset(lay[1]);
  const int stride = std::max(1, 1 << std::max(0, t.L - t.LH));
  const int smask = stride - 1;  // stride is a power of two: v mod stride = v & smask, also for v < 0
  const int64_t nint = grid_interior(N);
  if (t.keep_exact) {
    t.exactL.assign((size_t)7 * nint, 0.0);
    t.exactD.assign((size_t)nint, 0.0);
  }
  // the stencil of R_t A R_t^T at an interior point: A with the couplings to
  // non-interior points removed (only cell-boundary points have any)
  auto stencil = [&](int x, int y, int z, double *A) {
    host_stencil(t, x, y, z, A);
    if (on_cell_boundary(N, x, y, z))
      for (int d = 0; d < 15; ++d)
        if (!in_interior(N, x + dir_dx(d), y + dir_dy(d), z + dir_dz(d))) A[d] = 0.0;
  };
  // variable coefficient: stencils of a whole face layer, 15 per point, rows
  // in order; row y of layer z starts at point (y - 1)(N - 1 - z) - (y - 1) y / 2
  const bool pre = !t.const_kappa;
  const int nworkers = pre ? std::max(1, std::min<int>(15, (int)std::thread::hardware_concurrency() - 1)) : 0;
  auto row_start = [&](int y, int z) { return (size_t)(y - 1) * (N - 1 - z) - (size_t)(y - 1) * y / 2; };
  std::vector<double> stn[2];
  auto assemble = [&](int z, int part, int parts) {
    std::vector<double> &buf = stn[z & 1];
    for (int y = 1 + part; y <= N - 2 - z; y += parts)
      for (int x = 1; x <= N - 1 - y - z; ++x) stencil(x, y, z, &buf[(row_start(y, z) + x - 1) * 15]);
  };
  if (pre) {
    const size_t cap = (size_t)(N - 3) * (N - 2) / 2 * 15;  // points of the largest layer (z = 1), x 15
    stn[0].assign(cap, 0.0);
    stn[1].assign(cap, 0.0);
    if (N - 3 >= 1) {
      std::vector<std::thread> w;
      for (int k = 0; k < nworkers; ++k) w.emplace_back(assemble, 1, k, nworkers);
      for (auto &th : w) th.join();
    }
  }
  const bool ilu = t.factor == ILU_FACTOR_ILU0;
  int64_t i = 0;
  for (int z = 1; z <= N - 3; ++z) {
    std::vector<std::thread> workers;  // the next layer's stencils, meanwhile
    if (pre && z + 1 <= N - 3)
      for (int k = 0; k < nworkers; ++k) workers.emplace_back(assemble, z + 1, k, nworkers);
    // No per-layer reset: the recursion reads non-interior neighbours only
    // at x = 0 or y = 0 (never written) or in layer 0 (the first buffer, never
    // written before layer 2 starts); every other neighbour it reads is an
    // interior point computed earlier, and entries left over from layer z - 2
    // lie beyond this layer's diagonal x + y = N - 1 - z, where nothing reads.
    std::vector<double> &cur = lay[z & 1];
    const std::vector<double> &prv = lay[(z - 1) & 1];
    ilu_status st = ILU_OK;
    for (int y = 1; y <= N - 2 - z && st == ILU_OK; ++y)
      for (int x = 1; x <= N - 1 - y - z; ++x, ++i) {
        double Aloc[15];
        const double *A = Aloc;
        if (pre) A = &stn[z & 1][(row_start(y, z) + x - 1) * 15];
        else stencil(x, y, z, Aloc);
        // neighbour factor rows p + d for d in D_l
        const double *nb[7];
        for (int d = 0; d < 7; ++d) {
          const std::vector<double> &buf = dir_dz(d) < 0 ? prv : cur;
          nb[d] = &buf[((size_t)(y + dir_dy(d)) * S + (x + dir_dx(d))) * 8];
        }
        // symmetric Gauss-Seidel keeps the first term of each recursion: the
        // neighbour's stored pivot is then its diagonal entry a(p+d, p+d)
        double Lp[7];
        for (int k = 0; k < 7; ++k) {
          const int d = pl.order[k];
          double v = A[d];
          if (ilu)
            for (int m = 0; m < pl.nterm[d]; ++m) {
              const int e = pl.e[d][m];
              v -= Lp[e] * nb[e][7] * nb[d][pl.f[d][m]];
            }
          Lp[d] = v / nb[d][7];
        }
        double Dp = A[kCentre];
        if (ilu)
          for (int d = 0; d < 7; ++d) Dp -= Lp[d] * Lp[d] * nb[d][7];
        if (!(Dp > 0.0)) {
          err = ilu ? "non-positive ILU(0) pivot" : "non-positive diagonal entry";
          st = ILU_ESINGULAR;
          break;
        }
        double *me = &cur[((size_t)y * S + x) * 8];
        for (int d = 0; d < 7; ++d) me[d] = Lp[d];
        me[7] = Dp;
        if (t.keep_exact) {
          for (int d = 0; d < 7; ++d) t.exactL[(size_t)d * nint + i] = Lp[d];
          t.exactD[i] = Dp;
        }
        if (t.boundary == ILU_BOUNDARY_V1 && on_cell_boundary(N, x, y, z)) {  // records in lexicographic order
          // V1 (Alg. 1): L^p_d, d in D_l, and the multiplicative inverse of the centre
          for (int d = 0; d < 7; ++d) t.bndL.push_back(Lp[d]);
          t.bndL.push_back(1.0 / Dp);
        }
        for (int f = 0; f < 8; ++f) {
          const int dx = f < 7 ? dir_dx(f) : 0, dy = f < 7 ? dir_dy(f) : 0, dz = f < 7 ? dir_dz(f) : 0;
          if (((x - 1 + dx) & smask) || ((y - 1 + dy) & smask) || ((z - 1 + dz) & smask)) continue;
          if (f < 7 && !in_interior(N, x + dx, y + dy, z + dz)) continue;
          samples[f].push_back({x, y, z, f < 7 ? Lp[f] : 1.0 / Dp});
        }
      }
    for (auto &th : workers) th.join();
    if (st != ILU_OK) return st;
  }
  return ILU_OK;
}

static void fit_one(const HostTet &t, const std::vector<Sample> &smp, double *coef) {
  const int M = t.M;
  const int m = (int)smp.size();
  const int rows = m + M;
  std::vector<double> A((size_t)rows * M, 0.0), rhs(rows, 0.0);
  double px[16], py[16], pz[16];
  for (int r = 0; r < m; ++r) {
    legendre_all(t.deg[0], 2 * t.h * smp[r].x - 1, px);
    legendre_all(t.deg[1], 2 * t.h * smp[r].y - 1, py);
    legendre_all(t.deg[2], 2 * t.h * smp[r].z - 1, pz);
    for (int i = 0; i <= t.deg[0]; ++i)
      for (int j = 0; j <= t.deg[1]; ++j)
        for (int k = 0; k <= t.deg[2]; ++k)
          A[(size_t)((i * (t.deg[1] + 1) + j) * (t.deg[2] + 1) + k) * rows + r] = px[i] * py[j] * pz[k];
    rhs[r] = smp[r].v;
  }
  const double lam = t.ridge * std::sqrt((double)std::max(m, 1));
  for (int c = 0; c < M; ++c) A[(size_t)c * rows + m + c] = lam;
  if (!householder_lsq(rows, M, A, rhs, coef)) std::fill(coef, coef + M, 0.0);
}

ilu_status host_setup(HostTet &t, const double P[12], int level, const ilu_coeff *coeff, const int deg[3],
                      int sample_level, double ridge, std::string &err) {
  if (level < 2 || level > 10) { err = "level must be in [2, 10]"; return ILU_EINVAL; }
  for (int c = 0; c < 3; ++c)
    if (deg[c] < 0 || deg[c] > 12) { err = "surrogate degree must be in [0, 12]"; return ILU_EINVAL; }
  for (int k = 0; k < 12; ++k)
    if (!std::isfinite(P[k])) { err = "macro-tetrahedron has non-finite coordinates"; return ILU_EINVAL; }
  t.L = level;
  t.N = 1 << level;
  t.h = 1.0 / t.N;
  std::memcpy(t.P, P, sizeof(double) * 12);
  t.coeff = coeff ? *coeff : ilu_coeff{ILU_COEFF_CONST, 1.0, 0.0, 0};
  if (t.coeff.kind < 0 || t.coeff.kind > 2) { err = "unknown coefficient kind"; return ILU_EINVAL; }
  if (!std::isfinite(t.coeff.c0) || !std::isfinite(t.coeff.amp)) { err = "non-finite coefficient"; return ILU_EINVAL; }
  t.const_kappa = t.coeff.kind == ILU_COEFF_CONST;
  if (t.const_kappa && !(t.coeff.c0 > 0)) { err = "kappa must be positive"; return ILU_EINVAL; }
  for (int c = 0; c < 3; ++c) t.deg[c] = deg[c];
  t.M = (deg[0] + 1) * (deg[1] + 1) * (deg[2] + 1);
  t.LH = sample_level >= 0 ? sample_level : std::min(level, 5);
  t.ridge = ridge >= 0 ? ridge : 1e-6;
  // degeneracy: |det J| against the cube of the longest edge
  double e[3][3], scale = 0.0;
  for (int m = 0; m < 3; ++m)
    for (int c = 0; c < 3; ++c) {
      e[m][c] = P[3 * (m + 1) + c] - P[c];
      scale = std::max(scale, std::fabs(e[m][c]));
    }
  const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                     e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
  if (!(std::fabs(det) > 1e-12 * scale * scale * scale)) { err = "degenerate macro-tetrahedron"; return ILU_EINVAL; }
  element_classes(t);
  if (!stencil_weights(t, err)) return ILU_EINVAL;
  if (!t.const_kappa) {
    const int64_t nn = grid_nodes(t.N);
    t.kappa.assign((size_t)nn, 0.0);
    auto work = [&](int z0, int z1) {
      for (int z = z0; z < z1; ++z)
        for (int y = 0; y <= t.N - z; ++y)
          for (int x = 0; x <= t.N - z - y; ++x) {
            double X[3];
            host_phys(t, x, y, z, X);
            t.kappa[grid_index(t.N, x, y, z)] = host_kappa(t.coeff, X);
          }
    };
    const int nth = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int k = 0; k < nth; ++k) {
      int a = (int)((int64_t)(t.N + 1) * k / nth), b = (int)((int64_t)(t.N + 1) * (k + 1) / nth);
      if (a < b) pool.emplace_back(work, a, b);
    }
    for (auto &th : pool) th.join();
    for (double v : t.kappa)
      if (!(v > 0) || !std::isfinite(v)) { err = "kappa must be positive and finite at every grid point"; return ILU_EINVAL; }
  }
  t.keep_exact = level <= 7;
  t.bndL.clear();
  t.bnd_rowoff.clear();
  if (t.boundary == ILU_BOUNDARY_V1) {
    const int64_t rows = num_rows(t.N);
    t.bnd_rowoff.assign((size_t)rows + 1, 0);
    int acc = 0;
    for (int z = 1; z <= t.N - 3; ++z)
      for (int y = 1; y <= t.N - 2 - z; ++y) {
        t.bnd_rowoff[(size_t)row_id(t.N, y, z)] = acc;
        acc += bnd_row_count(t.N, y, z);
      }
    t.bnd_rowoff[(size_t)rows] = acc;
    t.bndL.reserve((size_t)acc * 8);
  }
  std::vector<Sample> samples[8];
  ilu_status st = factorise(t, samples, err);
  if (st != ILU_OK) return st;
  t.coefs.assign((size_t)8 * t.M, 0.0);
  {
    std::vector<std::thread> pool;
    for (int f = 0; f < 8; ++f) pool.emplace_back([&, f] { fit_one(t, samples[f], &t.coefs[(size_t)f * t.M]); });
    for (auto &th : pool) th.join();
  }
  build_row_tables(t);
  return ILU_OK;
}

}  // namespace ilu
