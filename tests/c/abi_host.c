/* A plain C99 client of include/ilu.h: host-only calls (no GPU).  Built and
 * run by tests/test_c_abi.py; prints one line per check and exits non-zero on
 * the first failure. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "ilu.h"

static int fails = 0;
#define CHECK(cond, what)                       \
  do {                                          \
    if (!(cond)) {                              \
      printf("FAIL %s (%s)\n", what, ilu_last_error()); \
      fails++;                                  \
    } else {                                    \
      printf("ok %s\n", what);                  \
    }                                           \
  } while (0)

int main(void) {
  /* grid helpers, Sec. 2.1 */
  CHECK(ilu_num_nodes(3) == 165, "num_nodes(3) = C(11,3)");
  CHECK(ilu_num_interior(4) == 455, "num_interior(4) = C(15,3)");
  CHECK(ilu_index(3, 0, 0, 0) == 0 && ilu_index(3, 0, 0, 8) == 164, "index of the corners");
  CHECK(ilu_index(3, 9, 0, 0) == -1, "index outside the grid");

  ilu_opts o;
  CHECK(ilu_opts_default(&o) == ILU_OK && o.precision == ILU_MIXED && o.device == 0, "opts_default");
  CHECK(ilu_opts_default(NULL) == ILU_EINVAL, "opts_default(NULL)");

  /* a host-only handle: set-up (Alg. 1, fit) without a device part */
  const double P[12] = {0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1};
  ilu_coeff k = {ILU_COEFF_CONST, 1.0, 0.0, 0};
  o.device = -1;
  ilu_tet t = NULL;
  CHECK(ilu_setup(P, 4, &k, 3, &o, &t) == ILU_OK && t != NULL, "setup host-only");
  double st[15];
  CHECK(ilu_stencil(t, 3, 3, 3, st) == ILU_OK, "stencil");
  double sum = 0.0;
  for (int d = 0; d < 15; ++d) sum += st[d];
  CHECK(fabs(sum) < 1e-12 && st[7] > 0.0, "stencil rows sum to zero, positive centre");
  double f[8];
  CHECK(ilu_exact_factor(t, 2, 2, 2, f) == ILU_OK && f[7] > 0.0, "exact factor");
  CHECK(ilu_smooth(t, NULL, NULL, 1, NULL, NULL) != ILU_OK, "smooth refuses a host-only handle");
  size_t n = ilu_surrogate_size(t);
  CHECK(n == 8 * 64, "surrogate size 8 x (3+1)^3");
  int perm[4];
  CHECK(ilu_vertex_order(t, perm) == ILU_OK && perm[0] == 0 && perm[3] == 3, "vertex order as given");
  CHECK(ilu_destroy(t) == ILU_OK, "destroy");

  /* local Fourier analysis, Sec. 3 */
  double mu = 0.0, all[24];
  CHECK(ilu_lfa_order(P, perm, &mu, all) == ILU_OK && mu > 0.0 && mu < 1.0, "lfa order");
  int best = 1;
  for (int i = 0; i < 24; ++i) best = best && all[i] >= mu * (1.0 - 1e-12); /* ties go to the first order */
  CHECK(best, "lfa picks the smallest factor");
  const double flat[12] = {0, 0, 0, 1, 0, 0, 2, 0, 0, 0, 0, 1};
  CHECK(ilu_lfa_order(flat, perm, &mu, NULL) == ILU_EINVAL, "lfa rejects a degenerate tet");

  /* argument errors */
  CHECK(ilu_setup(P, 11, &k, 3, &o, &t) == ILU_EINVAL, "level out of range");
  o.boundary = 7;
  CHECK(ilu_setup(P, 4, &k, 3, &o, &t) == ILU_EINVAL, "unknown boundary variant");
  o.boundary = ILU_BOUNDARY_V2;
  o.values = ILU_VALUES_TABULATED; /* an FP64 option */
  CHECK(ilu_setup(P, 4, &k, 3, &o, &t) == ILU_EINVAL, "tabulated values rejected for MIXED");
  o.precision = ILU_F64;
  CHECK(ilu_setup(P, 4, &k, 3, &o, &t) == ILU_OK && t != NULL, "tabulated values accepted for F64");
  ilu_destroy(t);
  t = NULL;
  /* batch calls refuse null arguments without touching a device */
  {
    int per_sweep = -1;
    CHECK(ilu_batch_launches(NULL, &per_sweep) == ILU_EINVAL && per_sweep == -1, "batch_launches(NULL batch)");
    CHECK(ilu_batch_create(NULL, 0, NULL, NULL) == ILU_EINVAL, "batch_create(NULL)");
  }
  /* the packed row schedule (host code): the level-8 plan runs on 640 lanes */
  {
    int nsteps = 0, lanes = 0;
    CHECK(ilu_packed_schedule(8, 1, 0, 0, &nsteps, &lanes, NULL, NULL) == ILU_OK && lanes == 640 &&
              nsteps % 8 == 0 && nsteps > 0,
          "level-8 packed schedule on 640 lanes");
    CHECK(ilu_packed_schedule(8, 1, 1017, 0, &nsteps, &lanes, NULL, NULL) == ILU_EINVAL, "more than 1016 lanes");
  }
  CHECK(strlen(ilu_version()) > 0, "version");
  return fails ? 1 : 0;
}
