/*
 * ilu.h -- C ABI of the GB300 matrix-free surrogate ILU(0) smoother.
 *
 * The operation is the smoother of Drzisga, Wagner and Wohlmuth, "A
 * matrix-free ILU realization based on surrogates" (arXiv 2210.15280):
 *
 *     x <- x + R_t^T (L~ D~ L~^T)^{-1} R_t (b - A x)          (Sec. 2.1, Alg. 2)
 *
 * on the interior points of one uniformly refined macro-tetrahedron t, where
 * A is the P1 stiffness matrix of -div(kappa grad u) (Sec. 2.1), L~ and D~ are
 * surrogate polynomials fitted to the exact ILU(0) factors of the interior
 * block (Sec. 3, Sec. 4.1, Alg. 1), evaluated on the fly in the sweep, and the
 * V2 boundary rule of Alg. 2 is used (L~^p_d = 0 where p+d is not interior).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.  level L in [2, 10], N = 2^L.  Logical grid G = {(x,y,z) in Z^3 :
 *   x,y,z >= 0, x+y+z <= N}, interior {x,y,z >= 1, x+y+z <= N-1} (Sec. 2.1).
 * Vectors.  Full-grid, lexicographic (z slowest, then y, then x; Sec. 2.1),
 *   length ilu_num_nodes(L) = (N+1)(N+2)(N+3)/6.  x entries on the boundary are
 *   Dirichlet data: read, never written.  b entries on the boundary are ignored.
 *   Element type: double for ILU_F64 and ILU_MIXED, float for ILU_F32.
 *   Device pointers unless the entry point says "host".  Vectors are owned by
 *   the caller; the handle owns its coefficients, tables and scratch.
 * Macro-tetrahedron.  12 doubles: vertices p1..p4 (x,y,z each).  The logical
 *   point (x,y,z) sits at p1 + ((p2-p1) x + (p3-p1) y + (p4-p1) z) / N.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls are asynchronous on it unless a host output is requested.
 * Errors.  Every entry point returns an ilu_status; no exception crosses the
 *   ABI.  ilu_last_error() gives a thread-local message for the last failure.
 *   ILU_ECUDA and ILU_ETIMEOUT leave the handle unusable: destroy it.
 * Devices.  A call may switch the calling thread to its handle's device while
 *   it runs; it puts the thread's current device back before it returns.
 */
#ifndef ILU_H
#define ILU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ILU_OK = 0,
  ILU_EINVAL = 1,     /* bad argument: level, degree, degenerate tet, null pointer, ... */
  ILU_ENOMEM = 2,     /* host or device allocation failed, or a memory budget is exceeded */
  ILU_ECUDA = 3,      /* a CUDA call failed; the handle is unusable */
  ILU_ESINGULAR = 4,  /* setup met a non-positive pivot or a non-positive surrogate 1/D */
  ILU_ENOTCONV = 5,   /* an iterative solve stopped at max_iter */
  ILU_ETIMEOUT = 6,   /* a bounded device wait ran out; the handle is unusable */
  ILU_EBUSY = 7,      /* the request loop is full or shutting down */
  ILU_ENODEV = 8      /* no CUDA device, or the handle has no device part */
} ilu_status;

typedef enum { ILU_F64 = 0, ILU_F32 = 1, ILU_MIXED = 2 } ilu_precision;

typedef enum {
  ILU_COEFF_CONST = 0,   /* kappa = c0 */
  ILU_COEFF_SINPROD = 1, /* kappa = c0 + amp sin(2 pi x) sin(2 pi y) sin(2 pi z) */
  ILU_COEFF_KAPPA_I = 2  /* kappa = 1 + 10 (x^i + y^i + z^i)  (Sec. 4.2) */
} ilu_coeff_kind;

/* Scalar diffusion coefficient kappa(x) of Sec. 2.1, evaluated at physical
 * points.  Element values are the mean of the four vertex values. */
typedef struct {
  int kind;   /* ilu_coeff_kind */
  double c0;  /* CONST / SINPROD offset */
  double amp; /* SINPROD amplitude */
  int ipow;   /* KAPPA_I exponent i */
} ilu_coeff;

/* Options.  Zero-initialise, then call ilu_opts_default. */
typedef struct {
  int deg[3];          /* surrogate degrees dg_x, dg_y, dg_z (Sec. 4.1); <0: use poly_degree */
  int sample_level;    /* coarse sampling level L_H (Sec. 4.1); <0: min(L, 5) */
  double ridge;        /* relative Tikhonov weight of the fit; <0: 1e-6 */
  int precision;       /* ilu_precision */
  int slabs;           /* z-slabs (CTAs) per tet in the sweep; <=0: automatic */
  int device;          /* CUDA device ordinal; -1: host-only handle (setup only) */
  long long max_wait_spins; /* bound on device-side spin waits; <=0: default */
  int kernel;          /* substitution kernels of FP32/MIXED sweeps: an ilu_kernel value */
  int factor;          /* factors the surrogates approximate: an ilu_factor value */
  int stencil;         /* how a variable-kappa operator is applied: an ilu_stencil_mode value */
  int orient;          /* vertex order used: an ilu_orient value */
  int boundary;        /* boundary variant of the factors: an ilu_boundary value */
  int max_cluster;     /* at most this many CTAs per cluster in the slab kernels; <=0: the largest the
                        * device schedules (lowest latency for one tet; smaller clusters pack more
                        * concurrent tets onto the GPU) */
  int values;          /* where FP64 substitutions take the surrogate values: an ilu_values_mode value */
} ilu_opts;

/* The two boundary variants of Sec. 4.1 and Alg. 2:
 *   ILU_BOUNDARY_V2  surrogates everywhere; a factor entry whose neighbour is
 *                    not interior is set to 0 in the substitutions (default);
 *   ILU_BOUNDARY_V1  at the interior points on the cell boundary (x = 1,
 *                    y = 1, z = 1 or x + y + z = N - 1) the exact ILU(0)
 *                    entries L^p_d, d in D_l, and 1/D^p computed by Alg. 1
 *                    at set-up are stored (8 values per such point, O(N^2)
 *                    in all) and used instead of the surrogates: L^p_d by
 *                    the forward substitution at p and by the backward one
 *                    wherever p - d is such a point, 1/D^p by the backward
 *                    one at p (Alg. 1 stores 1/beta_c for V1 and Sec. 4.1
 *                    has the stored stencils used by both substitutions).
 *                    Either substitution kernel family. */
typedef enum { ILU_BOUNDARY_V2 = 0, ILU_BOUNDARY_V1 = 1 } ilu_boundary;

/* Which vertex order of the macro-tetrahedron the handle uses (Sec. 3):
 *   ILU_ORIENT_GIVEN  p1..p4 as passed (default);
 *   ILU_ORIENT_LFA    the order ilu_lfa_order picks.  The logical grid, and
 *                     with it the layout of every vector, is then that of the
 *                     reordered tet: ilu_vertex_order tells which.
 * The ILU(0) smoother depends on the order (the lexicographic order of the
 * points follows the vertices); symmetric Gauss-Seidel does too. */
typedef enum { ILU_ORIENT_GIVEN = 0, ILU_ORIENT_LFA = 1 } ilu_orient;

/* How the residual applies A when kappa varies (constant kappa always uses
 * its 15 constants).  The paper computes the residual by assembling A or by
 * evaluating a surrogate of it (Sec. 4.1, residual step of Alg. 2):
 *   ILU_STENCIL_ON_THE_FLY  assemble each row in the residual from kappa at
 *                           the 15 neighbours (edge-star weights; about 230
 *                           FP64 flops per point, no storage);
 *   ILU_STENCIL_STORED      assemble the 14 off-diagonal coefficients of
 *                           every interior row once at set-up, in FP64 on the
 *                           device (14 x 8 bytes per grid point; FP32 for F32
 *                           sweeps), and read them in the residual;
 *   ILU_STENCIL_AUTO        stored when that array takes at most 4 GiB
 *                           (level 9 and below), otherwise on the fly.
 * In F64 and MIXED both give bit-identical residuals: the stored
 * coefficients are the same FP64 sums, applied in the same order.  F32
 * sweeps store the coefficients in FP32 (14 x 4 bytes per point) and apply
 * them in FP32, the precision of their residual. */
typedef enum { ILU_STENCIL_AUTO = 0, ILU_STENCIL_ON_THE_FLY = 1, ILU_STENCIL_STORED = 2 } ilu_stencil_mode;

/* Where the FP64 substitutions take the surrogate values L~^p_d and
 * 1/D~^p (Alg. 2 evaluates the polynomials at every point):
 *   ILU_VALUES_ON_THE_FLY  evaluate the row polynomials at every point inside
 *                          the substitutions (no storage beyond the row
 *                          tables);
 *   ILU_VALUES_TABULATED   evaluate them once for every grid point at set-up
 *                          (again after ilu_import_surrogate), on the device
 *                          with the same FP64 steps, and read them in the
 *                          substitutions: 2 x 64 bytes per grid point.
 *                          Levels <= 9;
 *   ILU_VALUES_AUTO        tabulated for F64 handles up to level 9 (the two
 *                          tables then take at most 2.9 GB); otherwise on
 *                          the fly.
 * The two give bit-identical sweeps.  The table trades memory for FP64
 * arithmetic: the substitutions are a chain of dependent hyperplane steps,
 * and on a GPU whose FP64 rate is a small fraction of its FP32 rate the
 * per-point polynomial evaluation dominates each step.  FP32 and MIXED
 * sweeps evaluate their FP32 polynomials on the fly (packed FP32 FMAs);
 * ILU_VALUES_TABULATED with them is ILU_EINVAL. */
typedef enum { ILU_VALUES_AUTO = 0, ILU_VALUES_ON_THE_FLY = 1, ILU_VALUES_TABULATED = 2 } ilu_values_mode;

/* Which L D L^T preconditioner the surrogates approximate (Sec. 4.2):
 *   ILU_FACTOR_ILU0  exact ILU(0) of the interior block, by Alg. 1 (default);
 *   ILU_FACTOR_SGS   symmetric Gauss-Seidel, the paper's comparison smoother:
 *                    L^p_d = A^p_d / A^{p+d}_c, D^p = A^p_c, i.e. the
 *                    factors of (D + E) D^-1 (D + E^T).
 * Sampling, fit, tables and sweeps are the same for both. */
typedef enum { ILU_FACTOR_ILU0 = 0, ILU_FACTOR_SGS = 1 } ilu_factor;

/* Substitution kernels of the FP32/MIXED sweeps.  All run the same
 * arithmetic (Alg. 2) and agree to rounding; they differ in how the
 * hyperplane wavefront is mapped onto the GPU:
 *   ILU_KERNEL_SLAB    a CTA per z-slab advancing one hyperplane per step with
 *                      block-wide synchronisation, slabs of a tet as clusters;
 *   ILU_KERNEL_BAND    a warp per (layer, 32-row band) advancing one row point
 *                      per lane and step, synchronised point to point through
 *                      tagged words (fastest from level 9 on);
 *   ILU_KERNEL_PACKED  one CTA per tet: its rows packed onto 384 lanes by a
 *                      host-computed schedule, one point per lane and step,
 *                      the CTA meeting at a block barrier after each step; no
 *                      CTA waits on another (levels up to 8, row degrees up to
 *                      6; fastest up to level 6, and the kernels to set up
 *                      tets with for batch throughput).
 * ILU_KERNEL_AUTO picks by level: packed up to 6, slab for 7 and 8, band from
 * 9.  F64 sweeps and degrees above 7 always use the slab kernels. */
typedef enum { ILU_KERNEL_AUTO = 0, ILU_KERNEL_SLAB = 1, ILU_KERNEL_BAND = 2, ILU_KERNEL_PACKED = 3 } ilu_kernel;

typedef struct ilu_tet_s *ilu_tet;
typedef struct ilu_batch_s *ilu_batch;
typedef struct ilu_server_s *ilu_server;

/* ---------------------------------------------------------------- setup -- */

/* Fill opts with defaults (deg -1, sample_level -1, ridge 1e-6, ILU_MIXED,
 * automatic slabs, device 0).  Returns ILU_EINVAL on NULL. */
ilu_status ilu_opts_default(ilu_opts *opts);

/* Set up the smoother for one macro-tetrahedron (Sec. 4.1, Alg. 1): assemble
 * the interior-restricted stencils, run the streaming LDL^T factorisation in
 * FP64 on the host, fit the eight surrogates (L_d for d in D_l, and 1/D_c) by
 * ridge-regularised least squares on the sample sets S_d, build the per-row
 * evaluation tables and upload them to `opts->device`.
 *   macro_tet   12 doubles (host), see conventions; must be non-degenerate.
 *   level       2..10.
 *   coeff       kappa (host); NULL means kappa = 1.
 *   poly_degree isotropic surrogate degree 0..10, used where opts->deg < 0.
 *   opts        NULL for defaults.
 *   out         receives the handle (NULL on failure).
 * Errors: ILU_EINVAL, ILU_ENOMEM, ILU_ESINGULAR, ILU_ECUDA, ILU_ENODEV. */
ilu_status ilu_setup(const double macro_tet[12], int level, const ilu_coeff *coeff, int poly_degree,
                     const ilu_opts *opts, ilu_tet *out);

/* Release the handle, its device memory and graphs.  NULL is accepted. */
ilu_status ilu_destroy(ilu_tet t);

/* Replace the fitted surrogate by externally supplied coefficients (same
 * layout as ilu_export_surrogate) and rebuild the evaluation tables (and the
 * tabulated values of an F64 handle).  Lets a caller run the sweep with
 * surrogates fitted elsewhere.  Synchronous; must not overlap a sweep of the
 * same handle on another stream.
 * Errors: ILU_EINVAL (count, non-finite value), ILU_ESINGULAR (1/D~ <= 0
 * somewhere; the previous coefficients stay), ILU_ECUDA (the upload failed:
 * the handle is marked failed). */
ilu_status ilu_import_surrogate(ilu_tet t, const double *coefs, size_t n);

/* Copy the surrogate coefficients to host memory: 8 blocks (w s se bnw bn bc
 * be, then 1/D) of (dgx+1)(dgy+1)(dgz+1) doubles, coefficient of
 * P_i(2hx-1) P_j(2hy-1) P_k(2hz-1) at index (i*(dgy+1)+j)*(dgz+1)+k, P_n the
 * Legendre polynomials and h = 2^-L.  n must be >= the block total. */
ilu_status ilu_export_surrogate(ilu_tet t, double *coefs, size_t n);

/* Number of doubles ilu_export_surrogate writes. */
size_t ilu_surrogate_size(ilu_tet t);

/* Host FP64 value of the surrogates at interior point (x,y,z), computed from
 * the same per-row tables the device uses: out[0..6] = L~^p_d for d in D_l
 * (V2-masked), out[7] = 1/D~^p.  Host only. */
ilu_status ilu_eval_surrogate(ilu_tet t, int x, int y, int z, double out[8]);

/* Host FP64 exact factor entries of Alg. 1 at interior point (x,y,z), kept
 * only when the handle was created at level <= 7: out[0..6] = L^p_d, out[7] =
 * D^p_c.  Returns ILU_EINVAL if not kept. */
ilu_status ilu_exact_factor(ilu_tet t, int x, int y, int z, double out[8]);

/* Host FP64 stencil A^p_d of the full operator at grid point (x,y,z) (all 15
 * directions in the order w s se bnw bn bc be c e n nw tse ts tc tw). */
ilu_status ilu_stencil(ilu_tet t, int x, int y, int z, double out[15]);

/* Local Fourier analysis of the ILU(0) smoother for the 24 vertex orders of
 * a macro-tetrahedron (Sec. 3): for each order, the constant stencil with
 * kappa = 1, its asymptotic ILU stencil (the stencil equations of Sec. 3,
 * Gauss-Seidel iteration from L_c = D_c = 1, L_d = 0), and the smoothing
 * factor mu = max |1 - A(t) / (L(t) D conj(L(t)))| over the high frequencies
 * of a 16^3 grid of (-pi, pi)^3 (t_k = -pi + 2 pi k / 16; at least one
 * component with |t| >= pi/2).
 *   perm    (host, out) perm[i] = index 0..3 of the vertex placed at
 *           position i by the order with the smallest mu (the first in
 *           lexicographic order among factors equal to 1e-12 relative).
 *   mu      (host, nullable) its factor.
 *   mu_all  (host, nullable, 24) the factors of all orders, lexicographic.
 * Host only.  ILU_EINVAL for a degenerate tet. */
ilu_status ilu_lfa_order(const double macro_tet[12], int perm[4], double *mu, double mu_all[24]);

/* The vertex order a handle uses: perm[i] = index of the caller's vertex at
 * position i (the identity unless set up with ILU_ORIENT_LFA). */
ilu_status ilu_vertex_order(ilu_tet t, int perm[4]);

/* ------------------------------------------------------------- smoothing -- */

/* `sweeps` applications of the smoother (Alg. 2) to device vectors x (in/out)
 * and b.  Each sweep: r = b - A x on the interior (FP64 in ILU_F64/MIXED,
 * FP32 in ILU_F32), forward substitution with L~, scaling by D~^-1 and
 * backward substitution with L~^T in the handle's precision, x += w.
 * res_norms (host, nullable, length sweeps) receives ||b - A x||_2 over the
 * interior before each sweep; giving it makes the call synchronous. */
ilu_status ilu_smooth(ilu_tet t, void *x, const void *b, int sweeps, void *stream, double *res_norms);

/* Same as ilu_smooth on HOST vectors: copies x and b to the device, smooths,
 * copies x back (synchronous). */
ilu_status ilu_smooth_host(ilu_tet t, void *x_host, const void *b_host, int sweeps, double *res_norms);

/* r = b - A x on the interior (boundary entries of r set to 0).  r (device,
 * nullable) has the handle's vector type; norm2 (host, nullable) receives
 * ||r||_2 and makes the call synchronous. */
ilu_status ilu_residual(ilu_tet t, const void *x, const void *b, void *r, double *norm2, void *stream);

/* r = b - A x and ||r||_2 like ilu_residual, for callers that cannot let a
 * library allocate device memory (a framework's caching allocator or a fixed
 * serving pool owns it, or cudaMalloc's implicit synchronisation is not
 * acceptable).  The paper has no counterpart.  The caller passes x, b (device,
 * the handle's vector type), r (device, same type; required; the call sets its
 * boundary entries to 0) and norm_dev (device, one double receiving ||r||_2).  The only
 * scratch, the per-block partial sums of the norm, lives in a fixed 1 MiB
 * device array inside the library: levels above 9 are rejected with
 * ILU_EINVAL.  The array is shared by all calls on a device and keeps the last
 * call's contents (every entry used is written before it is read); calls whose
 * kernels overlap on the GPU race on it and must be serialised. Host-only
 * handles are refused with ILU_ENODEV and failed ones with ILU_ECUDA, as
 * everywhere; the call holds the handle's lock while it launches.  The first
 * call on a device looks up the array's device address; make that first call
 * before any stream capture.  Asynchronous on `stream`; calls no allocator. */
ilu_status ilu_residual_noalloc(ilu_tet t, const void *x, const void *b, void *r, double *norm_dev, void *stream);

/* Outer iterations.  ilu_solve takes ILU_RICHARDSON or ILU_PCG; ilu_mg_solve
 * takes those two (V-cycle iteration, V-cycle-preconditioned CG) or their
 * multigrid names; a request of the request loop takes all four, the last two
 * selecting a resident multigrid hierarchy instead of a single tet. */
typedef enum { ILU_RICHARDSON = 0, ILU_PCG = 1, ILU_MG_VCYCLE = 2, ILU_MG_PCG = 3 } ilu_method;

/* Solve A x = b on the interior (boundary of x = Dirichlet data) to
 * ||b - A x||_2 <= rtol ||b||_2 (interior norms) with smoothed Richardson
 * (defect correction, x += C~^-1 r) or CG preconditioned by C~ (Sec. 4.2).
 * Residuals and updates are FP64 unless the handle is ILU_F32.
 * iters/rel_res (host, nullable) receive the iteration count and the final
 * relative residual.  Synchronous.  ILU_ENOTCONV at max_iter. */
ilu_status ilu_solve(ilu_tet t, void *x, const void *b, int method, double rtol, int max_iter, void *stream,
                     int *iters, double *rel_res);

/* The row schedule the packed kernels (ILU_KERNEL_PACKED) follow for one
 * substitution at a level (the same for every tet of that level), for
 * inspection and testing.  lanes: 0 for the kernels' own lane count (384 up
 * to level 7, 640 -- two CTAs of 320 -- at level 8), else 1..1016 for the
 * same construction on that many lanes; quantum: 0 for the
 * kernels' start quantum at that level (1 up to level 6, 2 at 7, 4 at 8),
 * else 1, 2 or 4.  *nsteps and *lanes_out receive its size; with entries and
 * lane_off (lanes + 1 ints) non-null they receive the schedule, rows grouped
 * by lane in step order, 8 ints per interior row, in the pass's own steps:
 *   [0] sw | (lo - sw) << 16 | far << 20: the row's switch step sw
 *       (quantum - 1 modulo the quantum; the lane computes no point there),
 *       the step lo of its first point, and bit j of far set if producer j
 *       is read from global memory;
 *   [1] n | y << 10 | z << 20, n the row's point count;
 *   [2] R0 | R1 << 15 and [3] R2 | row id << 15: R_j the word of the shared
 *       ring (lanes + 8 words a step; in a cluster every CTA holds all of
 *       it) holding producer j's value read at the first step of the 8-step
 *       block holding sw (word `lanes`, never written, if the producer row
 *       does not exist or is read from global memory);
 *   [4] the row coordinate (2x - (N - y - z)) / (2N) of step sw's point
 *       (float bits; x = 0 forward, n + lo - sw backward);
 *   [5..7] the producer codes: mode in bits 30-31 (0 no such interior row,
 *       1 read from the ring, 2 read from global memory), the producer's lane
 *       in bits 0-9, and in bits 10-29 the step distance k0 of the first value
 *       the consumer reads (the producer's value at step tau + 1 - k0 is its
 *       second value at step tau).
 * Forward producers of row (y, z): (y-1, z), (y, z-1), (y+1, z-1); backward:
 * (y+1, z), (y, z+1), (y-1, z+1).  Host-only; the paper sweeps
 * lexicographically on one core, this arrangement is the library's.
 * ILU_EINVAL for a level outside 2..8 or a bad lanes or quantum. */
ilu_status ilu_packed_schedule(int level, int forward, int lanes, int quantum, int *nsteps, int *lanes_out,
                               int *entries, int *lane_off);

/* Split n macro-tetrahedra over nranks GPUs for a batch or a request stream
 * on several devices: cost[i] (host, finite, >= 0; e.g. interior points x
 * sweeps) is tet i's work, rank_of[i] (host) receives its GPU.  Longest
 * processing time first: tets by decreasing cost, each to the least loaded
 * rank so far (ties to the lower rank, equal costs in index order); the
 * largest load stays within 4/3 of the optimum.  load (host, nullable,
 * nranks) receives each rank's total.  Interior solves on different tets are
 * independent (Sec. 2.1: the interface data are read, never written), so the
 * shards need no exchange.  Host-only; the paper runs one macro-primitive per
 * process, the split is this library's.  ILU_EINVAL for n < 0, nranks < 1,
 * null arrays or a bad cost. */
ilu_status ilu_partition(int n, const double *cost, int nranks, int *rank_of, double *load);

/* The dependency-depth floor of a substitution step on this GPU, for
 * roofline reporting: one CTA of `threads` threads (a multiple of 32, up to
 * 1024) runs `steps` steps of the shortest body a wavefront step can have --
 * three neighbour values from a shared-memory ring, seven dependent FMAs, the
 * result written back, a block barrier -- and *cycles_per_step receives the
 * SM cycles per step (best of two timed runs).  Alg. 2's substitutions are
 * chains of 3N - 11 such hyperplane steps (Sec. 2.1); steps x this floor
 * bounds any schedule that synchronises by block barrier.  ILU_ENODEV
 * without that device.  The paper has no counterpart. */
ilu_status ilu_step_floor(int device, int threads, int steps, double *cycles_per_step);

/* ----------------------------------------------------------------- batch -- */

/* Group tets for smoothing together.  All tets must live on one device and
 * share one precision; levels and degrees may differ.  Each tet runs on the
 * substitution kernels its own handle uses, so that it gets its single-tet
 * sweep bit for bit: tets on the packed kernels (the FP32/MIXED default up to
 * level 8) in one launch per row-table layout, a CTA per tet, most steps
 * first; the others on the slab kernels, grouped by level.  opts (nullable)
 * may set max_wait_spins and slabs: > 0 fixes the slab partition of every
 * slab tet (as in ilu_setup); otherwise the batch autotunes it, timing one
 * pass of the batch for each candidate (layers per slab CTA 1, 2, 4 x cluster
 * size for most resident CTAs or largest) on scratch vectors and keeping the
 * fastest.  The batch
 * keeps references to the tets, which must outlive it; it reuses each tet's
 * scratch, so a tet must not be smoothed by another call while a batch call
 * on it runs.  ILU_EINVAL for an empty batch, a null or failed tet, or mixed
 * devices or precisions.  The paper smooths one macro-tet at a time; batching
 * is this library's. */
ilu_status ilu_batch_create(const ilu_tet *tets, int n, const ilu_opts *opts, ilu_batch *out);
ilu_status ilu_batch_destroy(ilu_batch b);

/* `sweeps` sweeps of Alg. 2 on every tet of the batch: x[i], b[i] (host
 * arrays of n device pointers) are tet i's full-grid vectors, as for
 * ilu_smooth.  A pass is one residual launch over all tets and, per group of
 * tets on the slab kernels with equal level and row layout, one forward and
 * one backward launch; per group of tets on the packed kernels with equal row
 * layout and start quantum, one launch of both substitutions, and after them
 * one update launch x += w over all packed tets; the groups' launches run
 * concurrently.  The passes are captured in a CUDA
 * graph on the first call (again when `sweeps` changes) and replayed on
 * `stream`.  Synchronises `stream` before returning, to report a timed-out
 * wait (ILU_ETIMEOUT, the batch is then failed and must be destroyed).
 * Results equal ilu_smooth on each tet, bit for bit. */
ilu_status ilu_batch_smooth(ilu_batch bt, void *const *x, const void *const *b, int sweeps, void *stream);

/* The number of kernels one sweep of ilu_batch_smooth launches (residual
 * launches, group launches and the packed update launch), into *per_sweep.
 * ILU_EINVAL for a null argument. */
ilu_status ilu_batch_launches(ilu_batch bt, int *per_sweep);

/* ------------------------------------------------------------- multigrid -- */

/* Geometric multigrid on one macro-tetrahedron (Sec. 4.2 numerical results):
 * the nested lattices of levels 2..level, a V-cycle with nu pre- and nu
 * post-smoothing sweeps of Alg. 2 on every level above 2 and an exact solve
 * on level 2, whose one interior point is solved by division.
 *   - Smoother: one surrogate handle per level 3..level, set up as
 *     ilu_setup(macro_tet, l, coeff, poly_degree, opts) would; opts (nullable)
 *     selects precision, kernel and factor (ILU(0), or the symmetric
 *     Gauss-Seidel comparison smoother) for all levels.
 *   - Grid transfer: prolongation is the coarse piecewise-linear function
 *     evaluated at the fine points (a fine point with all coordinates even
 *     takes the coarse value; any other is the midpoint 2c + d of the coarse
 *     edge (c, c + d), d in D, and takes the mean of the two end values).
 *     Restriction is its transpose: b_c = r(2c) + (1/2) sum_{d in D} r(2c + d).
 *     Coarse operators are those of the coarse lattices, which equal the
 *     Galerkin products for constant kappa.
 * level in [3, 10], nu in [1, 16].  The handle owns one vector triple per
 * level (x, b, r in the vector type) and the level handles.  Errors as for
 * ilu_setup; ILU_EINVAL also for nu or level out of range.  The paper's
 * outer solvers (Steklov-Poincare iterations over macro-tets) are not part
 * of this library. */
typedef struct ilu_mg_s *ilu_mg;
ilu_status ilu_mg_setup(const double macro_tet[12], int level, const ilu_coeff *coeff, int poly_degree, int nu,
                        const ilu_opts *opts, ilu_mg *out);
ilu_status ilu_mg_destroy(ilu_mg mg);

/* Borrow the smoother handle of one level (3..finest), e.g. to export or
 * import its surrogate.  It stays owned by mg; do not destroy it. */
ilu_status ilu_mg_level(ilu_mg mg, int level, ilu_tet *out);

/* `cycles` V-cycles for A x = b on the finest level: x (in/out) and b as for
 * ilu_smooth.  res_norms (host, nullable, length cycles) receives ||b - A x||_2
 * over the interior after each cycle and makes the call synchronous. */
ilu_status ilu_mg_cycle(ilu_mg mg, void *x, const void *b, int cycles, void *stream, double *res_norms);

/* Solve A x = b to ||b - A x||_2 <= rtol ||b||_2 by V-cycle iteration
 * (ILU_RICHARDSON: x <- x + V(b - A x)) or by CG preconditioned with one
 * V-cycle from zero (ILU_PCG; symmetric since the smoother is symmetric, pre
 * and post counts are equal and restriction is the transposed prolongation).
 * Synchronous; ILU_ENOTCONV at max_iter. */
ilu_status ilu_mg_solve(ilu_mg mg, void *x, const void *b, int method, double rtol, int max_iter, void *stream,
                        int *iters, double *rel_res);

/* Asymptotic convergence factor of the V-cycle (Sec. 4.2): a power iteration
 * of `steps` cycles on the error propagation operator (b = 0) from the start
 * error e (device, full grid, boundary entries 0; overwritten), normalised
 * after every cycle.  rho (host) receives the last ratio of successive
 * interior norms; history (host, nullable, length steps) all of them.
 * Synchronous. */
ilu_status ilu_mg_rate(ilu_mg mg, void *e, int steps, void *stream, double *rho, double *history);

/* ----------------------------------------------------------- request loop -- */

typedef struct {
  double hbm_budget_bytes; /* device bytes the loop may hold for requests; <=0: 80% of free */
  int max_slots;           /* requests on the device at once; <=0: 64 */
  int device;
  int precision;           /* ilu_precision for admitted work */
  int max_cluster;         /* ilu_opts.max_cluster of the requests' set-ups; <=0: the library default */
} ilu_server_opts;

typedef struct {
  double macro_tet[12];
  int level;
  ilu_coeff coeff;
  int poly_degree;
  int method;        /* ilu_method; ILU_MG_VCYCLE / ILU_MG_PCG: V(3,3) multigrid, level >= 3 */
  double rtol;
  int max_iter;
  const double *b;   /* host, full grid, ilu_num_nodes(level) doubles; copied on submit */
  const double *x0;  /* host, nullable (zeros): start vector and Dirichlet data */
  int orient;        /* ilu_orient of the set-up (ILU_ORIENT_LFA: b, x0 and x in the reordered layout) */
  int boundary;      /* ilu_boundary of the set-up */
} ilu_request;

typedef struct {
  ilu_status status;
  int iters;
  double rel_res;
  double latency_ms;  /* submit to completion */
  double *x;          /* host solution, owned by the server until ilu_server_release */
  size_t n;
} ilu_result;

typedef struct {
  long long submitted, completed, failed;
  double p50_ms, p99_ms, solves_per_s;
  int max_concurrent;
} ilu_stats;

ilu_status ilu_server_create(const ilu_server_opts *opts, ilu_server *out);
/* Queue a request; returns at once with a ticket.  ILU_EBUSY if shutting down. */
ilu_status ilu_server_submit(ilu_server s, const ilu_request *req, uint64_t *ticket);
/* Wait up to timeout_ms (<0: forever) for a ticket.  ILU_ETIMEOUT if not done. */
ilu_status ilu_server_wait(ilu_server s, uint64_t ticket, int timeout_ms, ilu_result *res);
/* Free the host solution of a finished ticket. */
ilu_status ilu_server_release(ilu_server s, uint64_t ticket);
ilu_status ilu_server_stats(ilu_server s, ilu_stats *st);
ilu_status ilu_server_destroy(ilu_server s);

/* --------------------------------------------------------------- tracing -- */

/* Per-kernel device timing of one handle.  With enable != 0 every kernel the
 * handle launches is bracketed by CUDA events on its stream; ilu_profile_read
 * synchronises, returns the accumulated milliseconds of the residual, forward
 * and backward kernels in ms[0..2], their launch count in *launches, and
 * clears the counters.  The paper has no counterpart (it profiles with
 * LIKWID); this is the library's own tracing. */
ilu_status ilu_profile_enable(ilu_tet t, int enable);
ilu_status ilu_profile_read(ilu_tet t, double ms[3], long long *launches);

/* ------------------------------------------------------------- utilities -- */

/* (N+1)(N+2)(N+3)/6 for N = 2^level; 0 for level out of [2, 10]. */
size_t ilu_num_nodes(int level);
/* (N-1)(N-2)(N-3)/6; 0 for level out of range. */
size_t ilu_num_interior(int level);
/* Lexicographic index of (x,y,z), or -1 if the point is not in G. */
long long ilu_index(int level, int x, int y, int z);
/* Thread-local message of the last failed call on this thread. */
const char *ilu_last_error(void);
/* Library version string. */
const char *ilu_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ILU_H */
