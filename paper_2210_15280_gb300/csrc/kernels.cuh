// kernels.cuh -- device-side data of one macro-tetrahedron and the launchers
// of the sweep kernels (arXiv 2210.15280, Alg. 2 with the V2 boundary rule).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "grid.h"

namespace ilu {

constexpr int kMaxSlabs = 256;

// Everything a kernel needs to know about one tet.  Plain old data so that it
// can live in a device array for batched launches.
struct DevTet {
  int L, N;
  double h;
  int dx;          // surrogate degree in x = row polynomial degree
  int rstride;     // coefficients per function in the row tables
  int nslabs;      // z-slabs (CTAs) per substitution
  int slab_layers; // layers per slab (one warp per layer)
  int const_kappa;
  const void *tabF;  // rows x 7 x rstride (float or double)
  const void *tabB;  // rows x 8 x rstride
  const double *kappa;  // kappa at every grid point (variable coefficient)
  void *w;           // scratch, full grid, element type of the sweep
  int *flags;        // 2 * nslabs progress words + 2 ticket counters
  double A15[15];    // constant stencil
  double Wstar[100]; // edge-star weights (variable coefficient)
};

struct LaunchStatus {
  int code;     // 0 ok, otherwise an ilu_status value
  int where;    // slab that gave up
  int level;    // level it was waiting for
  int pad;
};

// precision of the sweep: W = element type of w and the row tables,
// X = element type of x and b, R = type the residual is computed in
enum SweepKind { kSweepF64 = 0, kSweepF32 = 1, kSweepMixed = 2 };

cudaError_t launch_residual(const DevTet &t, int kind, const void *x, const void *b, void *r_out, double *partials,
                            int nblocks_cap, int *nblocks_used, cudaStream_t st);
cudaError_t launch_norm_finish(const double *partials, int n, double *out, cudaStream_t st);
cudaError_t launch_forward(const DevTet &t, int kind, LaunchStatus *status, long long max_spins, cudaStream_t st);
cudaError_t launch_backward(const DevTet &t, int kind, void *x, LaunchStatus *status, long long max_spins,
                            cudaStream_t st);
cudaError_t launch_zero_interior_copy(const DevTet &t, int kind, const void *src, void *dst, cudaStream_t st);
size_t sweep_smem_bytes(int N, int slab_layers, int kind);
int residual_blocks(int N);

}  // namespace ilu
