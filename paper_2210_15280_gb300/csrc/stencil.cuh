// stencil.cuh -- the operator row of one interior point for a variable
// coefficient, applied to x without materialising the 15 coefficients.
//
// With kappa_T the mean of kappa at the four vertices of micro-tet T (Sec. 2.1),
// the coefficient of direction d is a fixed combination of kappa at the
// point's 15 stencil neighbours: A_d = sum over the edge-star pairs (d, q) of
// W[e] kappa(p + q) (grid.h lists the pairs, grouped by direction).  Rows sum
// to zero, so (A x)_p = sum_{d != c} A_d (x_{p+d} - x_p).  Each A_d is summed
// and applied at once, in the pair order, so only one coefficient is live.
#pragma once
#include <utility>

#include "grid.h"

namespace ilu {

ILU_HDC int star_begin(int d) {
  int e = 0;
  while (e < kStarPairs && star_d(e) < d) ++e;
  return e;
}

template <int B, int... I>
__device__ __forceinline__ double star_sum(std::integer_sequence<int, I...>, const double *kq, const double *W) {
  double a = 0.0;
  ((a = fma(W[B + I], kq[star_q(B + I)], a)), ...);
  return a;
}

template <typename TR, int D>
__device__ __forceinline__ void star_apply(TR &res, const double *kq, const TR *xv, const double *W, double xc) {
  if constexpr (D != kCentre) {
    constexpr int b = star_begin(D), e = star_begin(D + 1);
    const double a = star_sum<b>(std::make_integer_sequence<int, e - b>{}, kq, W);
    res = (TR)fma(-a, (double)xv[D] - xc, (double)res);
  }
}

// A_d of one direction alone
template <int D>
__device__ __forceinline__ double star_coeff(const double *kq, const double *W) {
  constexpr int b = star_begin(D), e = star_begin(D + 1);
  return star_sum<b>(std::make_integer_sequence<int, e - b>{}, kq, W);
}

// plane of direction d in the stored operator (the centre has none)
ILU_HDC int store_plane(int d) { return d < kCentre ? d : d - 1; }

template <typename TA, int... D>
__device__ __forceinline__ void star_store_all(std::integer_sequence<int, D...>, const double *kq, const double *W,
                                               TA *A, int64_t stride, int64_t i) {
  ((D != kCentre ? (void)(A[store_plane(D) * stride + i] = (TA)star_coeff<D>(kq, W)) : (void)0), ...);
}

// FP64 residuals (F64, MIXED): the same application as star_apply_all with
// the coefficients read from the stored planes, so identical operands in
// identical order give an identical result.  FP32 residuals (F32 sweeps):
// FP32 planes and FP32 arithmetic, the precision those sweeps work in.
__device__ __forceinline__ void stored_apply(double &res, const void *Av, int64_t stride, int64_t i, const double *xv) {
  const double *__restrict__ A = static_cast<const double *>(Av);
  const double xc = xv[kCentre];
#pragma unroll
  for (int d = 0; d < kNumDirs; ++d) {
    if (d == kCentre) continue;
    res = fma(-A[store_plane(d) * stride + i], xv[d] - xc, res);
  }
}
__device__ __forceinline__ void stored_apply(float &res, const void *Av, int64_t stride, int64_t i, const float *xv) {
  const float *__restrict__ A = static_cast<const float *>(Av);
  const float xc = xv[kCentre];
#pragma unroll
  for (int d = 0; d < kNumDirs; ++d) {
    if (d == kCentre) continue;
    res = fmaf(-A[store_plane(d) * stride + i], xv[d] - xc, res);
  }
}

template <typename TR, int... D>
__device__ __forceinline__ void star_apply_all(std::integer_sequence<int, D...>, TR &res, const double *kq,
                                               const TR *xv, const double *W) {
  const double xc = (double)xv[kCentre];
  (star_apply<TR, D>(res, kq, xv, W, xc), ...);
}

}  // namespace ilu
