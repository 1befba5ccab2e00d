// lfa.cpp -- vertex order of a macro-tetrahedron by local Fourier analysis
// of the ILU(0) smoother (arXiv 2210.15280, Sec. 3, after the stencil
// equations).
//
// For each of the 24 orders of the four vertices:
//   1. the constant stencil A_d of the reordered tet with kappa = 1;
//   2. the asymptotic ILU stencil: the stencil equations of Sec. 3 with the
//      same value at every point, iterated Gauss-Seidel fashion from
//      L_c = D_c = 1 and L_d = 0 until the values stop changing;
//   3. the symbols L(t) = 1 + sum_{d in D_l} L_d e^{i d.t}, D(t) = D_c and
//      A(t) = sum_{d in D} A_d e^{i d.t};
//   4. the smoothing factor, max |1 - A(t) / (L(t) D conj(L(t)))| over the
//      high frequencies of a 16^3 grid (t_k = -pi + 2 pi k / 16, at least one
//      component with |t| >= pi/2).
// The order with the smallest factor wins (the first in lexicographic order
// among factors equal to within 1e-12 relative, as symmetric shapes give).  Host code; a few milliseconds per tet.
#include <cmath>
#include <complex>
#include <cstring>
#include <string>

#include "../../include/ilu.h"
#include "grid.h"
#include "setup.h"

namespace ilu {
void set_last_error(const std::string &msg);
}

using namespace ilu;

namespace {

enum { W = 0, S, SE, BNW, BN, BC, BE, C };

// asymptotic L (directions w s se bnw bn bc be) and D of a constant stencil.
// The iteration runs on the stencil scaled to a unit diagonal: L is
// scale-free and D scales with A (the remark at the end of Sec. 3), and from
// the starting values L_c = D_c = 1 the iteration converges on that scale
// whatever the level A was assembled on.
void asymptotic(const double Ain[15], double L[7], double &D) {
  double A[15];
  for (int d = 0; d < 15; ++d) A[d] = Ain[d] / Ain[C];
  for (int k = 0; k < 7; ++k) L[k] = 0.0;
  D = 1.0;
  for (int it = 0; it < 5000; ++it) {
    double old[8];
    std::memcpy(old, L, sizeof(double) * 7);
    old[7] = D;
    L[BC] = A[BC] / D;
    L[S] = (A[S] - L[BC] * D * L[BN]) / D;
    L[BNW] = (A[BNW] - L[BC] * D * L[SE]) / D;
    L[BE] = (A[BE] - L[BC] * D * L[W]) / D;
    L[W] = (A[W] - L[BC] * D * L[BE] - L[BNW] * D * L[BN] - L[S] * D * L[SE]) / D;
    L[BN] = (A[BN] - L[BC] * D * L[S] - L[BE] * D * L[SE] - L[BNW] * D * L[W]) / D;
    L[SE] = (A[SE] - L[BC] * D * L[BNW] - L[BE] * D * L[BN] - L[S] * D * L[W]) / D;
    double q = 1.0;
    for (int k = 0; k < 7; ++k) q += L[k] * L[k];
    D = A[C] / q;
    double ch = std::fabs(D - old[7]);
    for (int k = 0; k < 7; ++k) ch = std::fmax(ch, std::fabs(L[k] - old[k]));
    if (ch <= 1e-15) break;
  }
  D *= Ain[C];
}

double smoothing_factor(const double A[15]) {
  double L[7], D;
  asymptotic(A, L, D);
  const int n = 16;
  const double pi = 3.14159265358979323846;
  double mu = 0.0;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c) {
        const double t[3] = {-pi + 2.0 * pi * a / n, -pi + 2.0 * pi * b / n, -pi + 2.0 * pi * c / n};
        if (std::fabs(t[0]) < pi / 2 && std::fabs(t[1]) < pi / 2 && std::fabs(t[2]) < pi / 2) continue;
        std::complex<double> Ls(1.0, 0.0), As(0.0, 0.0);
        for (int d = 0; d < kNumDirs; ++d) {
          const double ph = dir_dx(d) * t[0] + dir_dy(d) * t[1] + dir_dz(d) * t[2];
          const std::complex<double> e(std::cos(ph), std::sin(ph));
          As += A[d] * e;
          if (d < kNumLower) Ls += L[d] * e;
        }
        const std::complex<double> M = Ls * D * std::conj(Ls);
        const double r = std::abs((M - As) / M);
        if (!(r <= mu)) mu = r;  // a NaN propagates
      }
  return mu;
}

}  // namespace

namespace ilu {
// lexicographic permutations of (0 1 2 3)
void lfa_perm(int k, int p[4]) {
  int items[4] = {0, 1, 2, 3};
  int f = 6;
  for (int i = 0; i < 4; ++i) {
    const int j = k / f;
    k %= f;
    p[i] = items[j];
    for (int m = j; m < 3 - i; ++m) items[m] = items[m + 1];
    if (i < 3) f /= (3 - i);
  }
}
}  // namespace ilu

extern "C" ilu_status ilu_lfa_order(const double macro_tet[12], int perm[4], double *mu, double mu_all[24]) {
  if (!macro_tet || !perm) {
    set_last_error("null argument");
    return ILU_EINVAL;
  }
  double best = 0.0;
  int kbest = -1;
  for (int k = 0; k < 24; ++k) {
    int p[4];
    lfa_perm(k, p);
    double Q[12];
    for (int i = 0; i < 4; ++i)
      for (int c = 0; c < 3; ++c) Q[3 * i + c] = macro_tet[3 * p[i] + c];
    double A[15];
    std::string err;
    if (!unit_stencil(Q, A, err)) {
      set_last_error(err);
      return ILU_EINVAL;
    }
    const double m = smoothing_factor(A);
    if (!std::isfinite(m)) {
      set_last_error("local Fourier analysis did not converge");
      return ILU_ESINGULAR;
    }
    if (mu_all) mu_all[k] = m;
    if (kbest < 0 || m < best * (1.0 - 1e-12)) {  // ties (to rounding) keep the earlier order
      best = m;
      kbest = k;
    }
  }
  lfa_perm(kbest, perm);
  if (mu) *mu = best;
  return ILU_OK;
}
