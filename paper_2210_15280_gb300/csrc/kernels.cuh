// kernels.cuh -- device-side data of one macro-tetrahedron and the launchers
// of the sweep kernels (arXiv 2210.15280, Alg. 2 with the V2 boundary rule).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "grid.h"

namespace ilu {

// Partition of a tet for one substitution: zb face layers per z-slab (CTA),
// wpl compute warps per layer, P slabs launched as clusters of csize CTAs;
// prog = first progress word of the slabs in the flag array, ticket = the
// ticket counter of the clusters.
struct WaveGeom {
  int zb, wpl, P, csize, prog, ticket;
};

// Everything a kernel needs to know about one tet.  Plain old data so that it
// can live in a device array for batched launches.
struct DevTet {
  int L, N;
  double h;
  int dx;          // surrogate degree in x = row polynomial degree
  int rstride;     // coefficients per function in the row tables (4, 8 or 16, zero padded)
  WaveGeom fwd, bwd;
  int const_kappa;
  const void *tabF;  // rows x 7 x rstride (float or double)
  const void *tabB;  // rows x 8 x rstride
  const double *kappa;  // kappa at every grid point (variable coefficient)
  void *w;           // scratch, full grid, element type of the sweep
  int *flags;        // progress words of the slabs and the two ticket counters
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
// With cluster_query set nothing is launched: it receives the largest cluster
// size the device can schedule for this tet's kernel.
cudaError_t launch_forward(const DevTet &t, int kind, LaunchStatus *status, long long max_spins, cudaStream_t st,
                           int *cluster_query = nullptr);
cudaError_t launch_backward(const DevTet &t, int kind, void *x, LaunchStatus *status, long long max_spins,
                            cudaStream_t st, int *cluster_query = nullptr);
size_t wave_smem_bytes(int N, const WaveGeom &g, int kind, int dxp, bool forward);
// FP32/MIXED sweeps of degree <= 7 keep each row's polynomials in registers
// (CTAs of at most 16 warps); otherwise they are read from shared memory.
bool wave_uses_registers(int kind, int dx);
int residual_blocks(int N);

// solver helpers on full-grid vectors (double if f64, else float)
constexpr int kDotPartials = 512;
cudaError_t launch_dot(bool f64, const void *a, const void *b, long long n, double *partials, double *out,
                       cudaStream_t st);
cudaError_t launch_axpy(bool f64, void *y, const void *x, double a, long long n, cudaStream_t st);
cudaError_t launch_xpay(bool f64, void *p, const void *z, double b, long long n, cudaStream_t st);
cudaError_t launch_copy(bool src_f64, bool dst_f64, const void *src, void *dst, long long n, cudaStream_t st);
cudaError_t launch_interior_norm(int N, bool f64, const void *v, double *partials, int cap, double *out,
                                 cudaStream_t st);

}  // namespace ilu
