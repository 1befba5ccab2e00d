/*
 * oracle.c -- plain, slow, obviously-correct CPU reference for the matrix-free
 * surrogate ILU(0) smoother of Drzisga, Wagner and Wohlmuth (arXiv 2210.15280).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; it is used by tests/, by __graft_entry__.smoke() and by the CPU
 * baseline leg of bench.py.  It shares no code, header or table with the
 * library under paper_2210_15280_gb300/.
 *
 * Everything is FP64 and single-threaded.  Each function names the passage of
 * the paper it follows.  Conventions (the paper's, Sec. 2.1):
 *   N = 2^L edge intervals; logical grid G = {x,y,z >= 0, x+y+z <= N};
 *   interior G° = {x,y,z >= 1, x+y+z <= N-1};
 *   lexicographic order: z slowest, then y, then x fastest (Sec. 2.1);
 *   stencil directions in the order of the paper's set D:
 *     w s se bnw bn bc be | c | e n nw tse ts tc tw
 *   the first seven form D_l; direction 8+k is the negative of direction k.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR 1
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Stencil direction vectors (x, y, z); b = z-1, t = z+1 (Sec. 2.1). */
static const int DIR[15][3] = {
    {-1, 0, 0},  /* w   */
    {0, -1, 0},  /* s   */
    {1, -1, 0},  /* se  */
    {-1, 1, -1}, /* bnw */
    {0, 1, -1},  /* bn  */
    {0, 0, -1},  /* bc  */
    {1, 0, -1},  /* be  */
    {0, 0, 0},   /* c   */
    {1, 0, 0},   /* e   */
    {0, 1, 0},   /* n   */
    {-1, 1, 0},  /* nw  */
    {1, -1, 1},  /* tse */
    {0, -1, 1},  /* ts  */
    {0, 0, 1},   /* tc  */
    {-1, 0, 1},  /* tw  */
};

int orc_dir(int k, int c) { return DIR[k][c]; }

/* ---------------------------------------------------------------- grid --- */

/* Number of points of G (Sec. 2.1), counted by brute force. */
long orc_num_nodes(int N) {
  long n = 0;
  for (int z = 0; z <= N; ++z)
    for (int y = 0; y <= N - z; ++y) n += N - z - y + 1;
  return n;
}

int orc_in_grid(int N, int x, int y, int z) {
  return x >= 0 && y >= 0 && z >= 0 && x + y + z <= N;
}

int orc_in_interior(int N, int x, int y, int z) {
  return x >= 1 && y >= 1 && z >= 1 && x + y + z <= N - 1;
}

/* Lexicographic index of (x,y,z) in G: all points with smaller z come first,
 * then those with equal z and smaller y, then smaller x (Sec. 2.1).  Counted
 * by explicit loops so that it is correct by inspection. */
long orc_index(int N, int x, int y, int z) {
  long k = 0;
  for (int zz = 0; zz < z; ++zz)
    for (int yy = 0; yy <= N - zz; ++yy) k += N - zz - yy + 1;
  for (int yy = 0; yy < y; ++yy) k += N - z - yy + 1;
  return k + x;
}

/* Table of row starts: rowstart[z*(N+1)+y] = orc_index(N,0,y,z). */
static long *row_table(int N) {
  long *t = (long *)malloc(sizeof(long) * (size_t)(N + 1) * (N + 1));
  if (!t) return NULL;
  long k = 0;
  for (int z = 0; z <= N; ++z)
    for (int y = 0; y <= N; ++y) {
      t[(long)z * (N + 1) + y] = k;
      if (y <= N - z) k += N - z - y + 1;
    }
  return t;
}

static long IDX(const long *rt, int N, int x, int y, int z) {
  return rt[(long)z * (N + 1) + y] + x;
}

/* Coordinates of every point of G in lexicographic order. */
int orc_coords(int N, int *xyz) {
  long k = 0;
  for (int z = 0; z <= N; ++z)
    for (int y = 0; y <= N - z; ++y)
      for (int x = 0; x <= N - z - y; ++x) {
        xyz[3 * k] = x; xyz[3 * k + 1] = y; xyz[3 * k + 2] = z; ++k;
      }
  return ORC_OK;
}

/* -------------------------------------------------------------- mesh --- */

/* Lattice basis whose Kuhn simplices are the micro-tetrahedra.  Their edge
 * vectors are e=(1,0,0), ts=(0,-1,1), bc=(0,0,-1) and their sums
 * tse, be, s, se, i.e. exactly the 14 non-centre directions of D
 * (Sec. 2.1, figure of stencil directions; Bey refinement). */
static const int KA[3] = {1, 0, 0}, KB[3] = {0, -1, 1}, KC[3] = {0, 0, -1};
static const int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

/* Enumerate all micro-tetrahedra: for each lattice point q and permutation s
 * of (a,b,c) the simplex {q, q+s0, q+s0+s1, q+a+b+c}; keep it if all four
 * vertices lie in G.  Writes 12 ints per tet if out != NULL; returns count. */
long orc_enumerate_tets(int N, int *out) {
  const int *V[3] = {KA, KB, KC};
  long n = 0;
  for (int qz = -1; qz <= N + 1; ++qz)
    for (int qy = -1; qy <= N + 1; ++qy)
      for (int qx = -1; qx <= N + 1; ++qx)
        for (int p = 0; p < 6; ++p) {
          int v[4][3];
          const int *s0 = V[PERM[p][0]], *s1 = V[PERM[p][1]];
          for (int c = 0; c < 3; ++c) {
            int q = c == 0 ? qx : (c == 1 ? qy : qz);
            v[0][c] = q;
            v[1][c] = q + s0[c];
            v[2][c] = q + s0[c] + s1[c];
            v[3][c] = q + KA[c] + KB[c] + KC[c];
          }
          int ok = 1;
          for (int i = 0; i < 4; ++i) ok &= orc_in_grid(N, v[i][0], v[i][1], v[i][2]);
          if (!ok) continue;
          if (out)
            for (int i = 0; i < 4; ++i)
              for (int c = 0; c < 3; ++c) out[12 * n + 3 * i + c] = v[i][c];
          ++n;
        }
  return n;
}

/* Physical position of logical point (x,y,z): base vertex plus the edge
 * vectors d_i = P_{i+1} - P_1 scaled by (x,y,z)/N (Sec. 2.1; the divisor is
 * read as 2^L so that the corner x = 2^L lands on the second macro vertex). */
void orc_phys(const double *P, int N, double x, double y, double z, double *X) {
  for (int c = 0; c < 3; ++c)
    X[c] = P[c] + ((P[3 + c] - P[c]) * x + (P[6 + c] - P[c]) * y + (P[9 + c] - P[c]) * z) / N;
}

/* Scalar coefficient kappa at a physical point.  kind 0: c0 (constant);
 * kind 1: c0 + amp*sin(2 pi x) sin(2 pi y) sin(2 pi z);
 * kind 2: 1 + 10 (x^i + y^i + z^i), the family of Sec. 4.2. */
double orc_kappa(int kind, double c0, double amp, int ipow, const double *X) {
  if (kind == 0) return c0;
  if (kind == 1) {
    const double tp = 2.0 * M_PI;
    return c0 + amp * sin(tp * X[0]) * sin(tp * X[1]) * sin(tp * X[2]);
  }
  return 1.0 + 10.0 * (pow(X[0], ipow) + pow(X[1], ipow) + pow(X[2], ipow));
}

/* P1 element stiffness of one tetrahedron with physical vertices X[4][3]:
 * K_ij = |T| kappa_T grad(phi_i) . grad(phi_j)  (Eq. for A_ij, Sec. 2.1),
 * kappa_T = mean of kappa at the four vertices.  Returns |T|. */
double orc_element(const double X[4][3], const double kv[4], double K[4][4]) {
  double E[3][3]; /* columns: X1-X0, X2-X0, X3-X0 */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) E[r][c] = X[c + 1][r] - X[0][r];
  double det = E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) -
               E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
               E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
  /* inverse of E: rows are the gradients of the barycentric functions 1..3 */
  double Ei[3][3];
  Ei[0][0] = (E[1][1] * E[2][2] - E[1][2] * E[2][1]) / det;
  Ei[0][1] = (E[0][2] * E[2][1] - E[0][1] * E[2][2]) / det;
  Ei[0][2] = (E[0][1] * E[1][2] - E[0][2] * E[1][1]) / det;
  Ei[1][0] = (E[1][2] * E[2][0] - E[1][0] * E[2][2]) / det;
  Ei[1][1] = (E[0][0] * E[2][2] - E[0][2] * E[2][0]) / det;
  Ei[1][2] = (E[0][2] * E[1][0] - E[0][0] * E[1][2]) / det;
  Ei[2][0] = (E[1][0] * E[2][1] - E[1][1] * E[2][0]) / det;
  Ei[2][1] = (E[0][1] * E[2][0] - E[0][0] * E[2][1]) / det;
  Ei[2][2] = (E[0][0] * E[1][1] - E[0][1] * E[1][0]) / det;
  double g[4][3];
  for (int c = 0; c < 3; ++c) {
    g[1][c] = Ei[0][c]; g[2][c] = Ei[1][c]; g[3][c] = Ei[2][c];
    g[0][c] = -(Ei[0][c] + Ei[1][c] + Ei[2][c]);
  }
  double vol = fabs(det) / 6.0;
  double kT = 0.25 * (kv[0] + kv[1] + kv[2] + kv[3]);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      K[i][j] = vol * kT * (g[i][0] * g[j][0] + g[i][1] * g[j][1] + g[i][2] * g[j][2]);
  return vol;
}

/* ------------------------------------------------------ global matrix --- */

#define ROWCAP 24

/* Assemble the global stiffness matrix on all of G by a loop over all
 * micro-tetrahedra (A_ij = a(phi_i, phi_j), Sec. 2.1).  Output is CSR with
 * sorted columns; rowptr has nn+1 entries, col/val have capacity cap.
 * Returns the number of nonzeros, or -1 if a row exceeds ROWCAP entries or
 * cap is too small. */
long orc_assemble(int N, const double *P, int kind, double c0, double amp, int ipow,
                  long *rowptr, long *col, double *val, long cap) {
  long nn = orc_num_nodes(N);
  long *rt = row_table(N);
  long *rc = (long *)malloc(sizeof(long) * nn * ROWCAP);
  double *rv = (double *)malloc(sizeof(double) * nn * ROWCAP);
  int *cnt = (int *)calloc(nn, sizeof(int));
  double *kap = (double *)malloc(sizeof(double) * nn);
  long ntet = orc_enumerate_tets(N, NULL);
  int *tets = (int *)malloc(sizeof(int) * 12 * ntet);
  long result = -1;
  if (!rt || !rc || !rv || !cnt || !kap || !tets) goto done;
  orc_enumerate_tets(N, tets);
  for (int z = 0; z <= N; ++z)
    for (int y = 0; y <= N - z; ++y)
      for (int x = 0; x <= N - z - y; ++x) {
        double X[3];
        orc_phys(P, N, x, y, z, X);
        kap[IDX(rt, N, x, y, z)] = orc_kappa(kind, c0, amp, ipow, X);
      }
  for (long t = 0; t < ntet; ++t) {
    double X[4][3], kv[4], K[4][4];
    long id[4];
    for (int i = 0; i < 4; ++i) {
      int *v = tets + 12 * t + 3 * i;
      orc_phys(P, N, v[0], v[1], v[2], X[i]);
      id[i] = IDX(rt, N, v[0], v[1], v[2]);
      kv[i] = kap[id[i]];
    }
    orc_element(X, kv, K);
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        long r = id[i];
        int f = -1;
        for (int m = 0; m < cnt[r]; ++m)
          if (rc[r * ROWCAP + m] == id[j]) { f = m; break; }
        if (f < 0) {
          if (cnt[r] >= ROWCAP) goto done;
          f = cnt[r]++;
          rc[r * ROWCAP + f] = id[j];
          rv[r * ROWCAP + f] = 0.0;
        }
        rv[r * ROWCAP + f] += K[i][j];
      }
  }
  long nz = 0;
  rowptr[0] = 0;
  for (long r = 0; r < nn; ++r) {
    /* insertion sort of the row by column */
    long *c = rc + r * ROWCAP;
    double *v = rv + r * ROWCAP;
    for (int a = 1; a < cnt[r]; ++a) {
      long ck = c[a]; double vk = v[a]; int b = a - 1;
      while (b >= 0 && c[b] > ck) { c[b + 1] = c[b]; v[b + 1] = v[b]; --b; }
      c[b + 1] = ck; v[b + 1] = vk;
    }
    if (nz + cnt[r] > cap) goto done;
    for (int m = 0; m < cnt[r]; ++m) { col[nz] = c[m]; val[nz] = v[m]; ++nz; }
    rowptr[r + 1] = nz;
  }
  result = nz;
done:
  free(rt); free(rc); free(rv); free(cnt); free(kap); free(tets);
  return result;
}

/* Local stencil of the full operator at one point p (all 15 directions),
 * assembled from the micro-tetrahedra that contain p.  Used where the global
 * matrix is too large to hold; tests check it against orc_assemble. */
int orc_local_stencil(int N, const double *P, int kind, double c0, double amp, int ipow,
                      int x, int y, int z, double *st) {
  const int *V[3] = {KA, KB, KC};
  for (int d = 0; d < 15; ++d) st[d] = 0.0;
  /* a tet containing p has p at one of its 4 local positions; its base q is
   * p minus that vertex's offset */
  for (int p = 0; p < 6; ++p) {
    const int *s0 = V[PERM[p][0]], *s1 = V[PERM[p][1]];
    int off[4][3];
    for (int c = 0; c < 3; ++c) {
      off[0][c] = 0; off[1][c] = s0[c]; off[2][c] = s0[c] + s1[c];
      off[3][c] = KA[c] + KB[c] + KC[c];
    }
    for (int loc = 0; loc < 4; ++loc) {
      int v[4][3], ok = 1;
      for (int i = 0; i < 4; ++i) {
        v[i][0] = x - off[loc][0] + off[i][0];
        v[i][1] = y - off[loc][1] + off[i][1];
        v[i][2] = z - off[loc][2] + off[i][2];
        ok &= orc_in_grid(N, v[i][0], v[i][1], v[i][2]);
      }
      if (!ok) continue;
      double X[4][3], kv[4], K[4][4];
      for (int i = 0; i < 4; ++i) {
        orc_phys(P, N, v[i][0], v[i][1], v[i][2], X[i]);
        kv[i] = orc_kappa(kind, c0, amp, ipow, X[i]);
      }
      orc_element(X, kv, K);
      for (int j = 0; j < 4; ++j) {
        int dd[3] = {v[j][0] - x, v[j][1] - y, v[j][2] - z};
        int found = -1;
        for (int d = 0; d < 15; ++d)
          if (DIR[d][0] == dd[0] && DIR[d][1] == dd[1] && DIR[d][2] == dd[2]) found = d;
        if (found < 0) return ORC_ERR;
        st[found] += K[loc][j];
      }
    }
  }
  return ORC_OK;
}

/* --------------------------------------------------------- exact ILU --- */

/* Interior numbering: intid[k] = position of grid point k among interior
 * points in lexicographic order, or -1 on the boundary.  Returns count. */
long orc_interior_ids(int N, long *intid) {
  long k = 0, m = 0;
  for (int z = 0; z <= N; ++z)
    for (int y = 0; y <= N - z; ++y)
      for (int x = 0; x <= N - z - y; ++x, ++k) intid[k] = orc_in_interior(N, x, y, z) ? m++ : -1;
  return m;
}

static long find_col(const long *col, long a, long b, long j) {
  while (a < b) {
    long m = (a + b) / 2;
    if (col[m] < j) a = m + 1; else b = m;
  }
  return a;
}

/* ILU(0) of the interior block A_tt = R_t A R_t^T (Sec. 3) by the textbook
 * IKJ variant of Gaussian elimination restricted to the sparsity pattern
 * (Saad, Iterative Methods for Sparse Linear Systems, Alg. 10.4).
 * In: full-grid CSR.  Out: for every interior point p (interior order) the
 * unit-lower factor entries L^p_d for d in D_l (0 where p+d is not interior)
 * and the pivot D^p_c, so that (L D L^T)_ij = (A_tt)_ij on the pattern.
 * Returns ORC_ERR on a non-positive pivot. */
int orc_ilu0(int N, const long *rowptr, const long *col, const double *val,
             double *Lout /* 7*nint, [d*nint+i] */, double *Dout) {
  long nn = orc_num_nodes(N);
  long *intid = (long *)malloc(sizeof(long) * nn);
  long nint = orc_interior_ids(N, intid);
  long *ip = (long *)malloc(sizeof(long) * (nint + 1));
  long *ic = (long *)malloc(sizeof(long) * rowptr[nn]);
  double *iv = (double *)malloc(sizeof(double) * rowptr[nn]);
  long *pts = (long *)malloc(sizeof(long) * nint);
  int rc = ORC_ERR;
  if (!intid || !ip || !ic || !iv || !pts) goto done;
  /* interior block in CSR (columns stay sorted since the numbering is monotone) */
  long nz = 0, r = 0;
  ip[0] = 0;
  for (long k = 0; k < nn; ++k) {
    if (intid[k] < 0) continue;
    pts[r] = k;
    for (long m = rowptr[k]; m < rowptr[k + 1]; ++m)
      if (intid[col[m]] >= 0) { ic[nz] = intid[col[m]]; iv[nz] = val[m]; ++nz; }
    ip[++r] = nz;
  }
  /* IKJ elimination */
  for (long i = 1; i < nint; ++i) {
    for (long mk = ip[i]; mk < ip[i + 1] && ic[mk] < i; ++mk) {
      long k = ic[mk];
      long dk = find_col(ic, ip[k], ip[k + 1], k);
      iv[mk] /= iv[dk];
      for (long mj = mk + 1; mj < ip[i + 1]; ++mj) {
        long j = ic[mj];
        long q = find_col(ic, ip[k], ip[k + 1], j);
        if (q < ip[k + 1] && ic[q] == j) iv[mj] -= iv[mk] * iv[q];
      }
    }
  }
  /* read off L (strictly lower part) and the pivots */
  int *xyz = (int *)malloc(sizeof(int) * 3 * nn);
  if (!xyz) goto done;
  orc_coords(N, xyz);
  long *rt = row_table(N);
  for (long i = 0; i < nint; ++i) {
    long g = pts[i];
    int x = xyz[3 * g], y = xyz[3 * g + 1], z = xyz[3 * g + 2];
    long dii = find_col(ic, ip[i], ip[i + 1], i);
    Dout[i] = iv[dii];
    if (!(Dout[i] > 0.0)) { free(xyz); free(rt); goto done; }
    for (int d = 0; d < 7; ++d) {
      int qx = x + DIR[d][0], qy = y + DIR[d][1], qz = z + DIR[d][2];
      double v = 0.0;
      if (orc_in_interior(N, qx, qy, qz)) {
        long j = intid[IDX(rt, N, qx, qy, qz)];
        long q = find_col(ic, ip[i], ip[i + 1], j);
        if (q < ip[i + 1] && ic[q] == j) v = iv[q];
      }
      Lout[(long)d * nint + i] = v;
    }
  }
  free(xyz); free(rt);
  rc = ORC_OK;
done:
  free(intid); free(ip); free(ic); free(iv); free(pts);
  return rc;
}

/* Symmetric Gauss-Seidel as an L D L^T preconditioner, the comparison
 * smoother of Sec. 4.2: with E the strictly lower part of A_tt in the
 * lexicographic order and D its diagonal, C = (D + E) D^{-1} (D + E^T) has the
 * unit-lower factor I + E D^{-1}, i.e. L^p_d = A(p, p+d) / A(p+d, p+d) (0 where
 * p+d is not interior), and the pivots D^p = A(p, p).
 * Out (interior order): L[d*nint+i] for d in D_l and D[i]. */
int orc_sgs_factors(int N, const long *rowptr, const long *col, const double *val, double *Lout, double *Dout) {
  long nn = orc_num_nodes(N);
  long *intid = (long *)malloc(sizeof(long) * nn);
  int *xyz = (int *)malloc(sizeof(int) * 3 * nn);
  long *rt = row_table(N);
  if (!intid || !xyz || !rt) { free(intid); free(xyz); free(rt); return ORC_ERR; }
  long nint = orc_interior_ids(N, intid);
  orc_coords(N, xyz);
  double *diag = (double *)malloc(sizeof(double) * nn);
  if (!diag) { free(intid); free(xyz); free(rt); return ORC_ERR; }
  for (long g = 0; g < nn; ++g) {
    diag[g] = 0.0;
    for (long m = rowptr[g]; m < rowptr[g + 1]; ++m)
      if (col[m] == g) diag[g] = val[m];
  }
  for (long g = 0; g < nn; ++g) {
    long i = intid[g];
    if (i < 0) continue;
    int x = xyz[3 * g], y = xyz[3 * g + 1], z = xyz[3 * g + 2];
    Dout[i] = diag[g];
    for (int d = 0; d < 7; ++d) {
      int qx = x + DIR[d][0], qy = y + DIR[d][1], qz = z + DIR[d][2];
      double v = 0.0;
      if (orc_in_interior(N, qx, qy, qz)) {
        long q = IDX(rt, N, qx, qy, qz);
        for (long m = rowptr[g]; m < rowptr[g + 1]; ++m)
          if (col[m] == q) v = val[m] / diag[q];
      }
      Lout[(long)d * nint + i] = v;
    }
  }
  free(intid); free(xyz); free(rt); free(diag);
  return ORC_OK;
}

/* One symmetric Gauss-Seidel sweep written out directly: over the interior
 * points in lexicographic order x_i <- (b_i - sum_{j != i} a_ij x_j) / a_ii
 * with the newest values, then the same in reverse order.  Boundary entries
 * of x are Dirichlet data and are not changed. */
int orc_sgs_sweep(int N, const long *rowptr, const long *col, const double *val, double *x, const double *b) {
  long nn = orc_num_nodes(N);
  long *intid = (long *)malloc(sizeof(long) * nn);
  if (!intid) return ORC_ERR;
  orc_interior_ids(N, intid);
  for (int pass = 0; pass < 2; ++pass)
    for (long k = 0; k < nn; ++k) {
      long g = pass == 0 ? k : nn - 1 - k;
      if (intid[g] < 0) continue;
      double s = b[g], a = 0.0;
      for (long m = rowptr[g]; m < rowptr[g + 1]; ++m) {
        if (col[m] == g) a = val[m];
        else s -= val[m] * x[col[m]];
      }
      x[g] = s / a;
    }
  free(intid);
  return ORC_OK;
}

/* ---------------------------------------------------------- Alg. 1 ---- */

/* Memory-efficient in-place LDL^T factorisation of Algorithm 1 (Sec. 4.1),
 * written in the paper's notation: beta holds the factorised stencils of the
 * current face layer, gamma those of the layer below.  The operator entries
 * are those of the interior-restricted matrix R_t A R_t^T (Sec. 3): zero
 * where p+d is not an interior point.  Stencils come from orc_local_stencil.
 * Out (interior order): L[d*nint+i] for d in D_l and D[i].
 * Memory is O(N^2) apart from the outputs. */
int orc_alg1(int N, const double *P, int kind, double c0, double amp, int ipow,
             double *Lout, double *Dout) {
  const int M = N + 2; /* layer arrays indexed (x+1, y+1) to allow x-1 = -1 */
  enum { W = 0, S, SE, BNW, BN, BC, BE, C };
  double *beta = (double *)malloc(sizeof(double) * 8 * M * M);
  double *gamma = (double *)malloc(sizeof(double) * 8 * M * M);
  if (!beta || !gamma) { free(beta); free(gamma); return ORC_ERR; }
#define B(d, x, y) beta[((d) * M + (x) + 1) * M + (y) + 1]
#define G(d, x, y) gamma[((d) * M + (x) + 1) * M + (y) + 1]
  for (int d = 0; d < 8; ++d)
    for (int i = 0; i < M * M; ++i) {
      beta[d * M * M + i] = d == C ? 1.0 : 0.0;
      gamma[d * M * M + i] = d == C ? 1.0 : 0.0;
    }
  long i = 0, nint = 0;
  for (int z = 1; z <= N - 1; ++z)
    for (int y = 1; y <= N - 1 - z; ++y) nint += (N - 1 - z - y > 0) ? N - 1 - z - y : 0;
  for (int z = 1; z <= N - 1; ++z) {
    for (int y = 1; y <= N - 1 - z; ++y) {
      for (int x = 1; x <= N - 1 - z - y; ++x, ++i) {
        double st[15], A[15];
        if (orc_local_stencil(N, P, kind, c0, amp, ipow, x, y, z, st) != ORC_OK) goto fail;
        for (int d = 0; d < 15; ++d)
          A[d] = orc_in_interior(N, x + DIR[d][0], y + DIR[d][1], z + DIR[d][2]) ? st[d] : 0.0;
        double bc = A[BC] / G(C, x, y);
        double s = (A[S] - bc * G(C, x, y) * B(BN, x, y - 1)) / B(C, x, y - 1);
        double bnw = (A[BNW] - bc * G(C, x, y) * G(SE, x - 1, y + 1)) / G(C, x - 1, y + 1);
        double be = (A[BE] - bc * G(C, x, y) * G(W, x + 1, y)) / G(C, x + 1, y);
        double w = (A[W] - bc * G(C, x, y) * B(BE, x - 1, y) - bnw * G(C, x - 1, y + 1) * B(BN, x - 1, y) -
                    s * B(C, x, y - 1) * B(SE, x - 1, y)) / B(C, x - 1, y);
        double bn = (A[BN] - bc * G(C, x, y) * G(S, x, y + 1) - be * G(C, x + 1, y) * G(SE, x, y + 1) -
                     bnw * G(C, x - 1, y + 1) * G(W, x, y + 1)) / G(C, x, y + 1);
        double se = (A[SE] - bc * G(C, x, y) * B(BNW, x + 1, y - 1) - be * G(C, x + 1, y) * B(BN, x + 1, y - 1) -
                     s * B(C, x, y - 1) * B(W, x + 1, y - 1)) / B(C, x + 1, y - 1);
        double c = A[C] - bc * bc * G(C, x, y) - be * be * G(C, x + 1, y) - bnw * bnw * G(C, x - 1, y + 1) -
                   bn * bn * G(C, x, y + 1) - se * se * B(C, x + 1, y - 1) - s * s * B(C, x, y - 1) -
                   w * w * B(C, x - 1, y);
        B(BC, x, y) = bc; B(S, x, y) = s; B(BNW, x, y) = bnw; B(BE, x, y) = be;
        B(W, x, y) = w; B(BN, x, y) = bn; B(SE, x, y) = se; B(C, x, y) = c;
        if (Dout) Dout[i] = c;
        if (Lout) { /* D_l order w s se bnw bn bc be, interior numbering i */
          Lout[0 * nint + i] = w; Lout[1 * nint + i] = s; Lout[2 * nint + i] = se;
          Lout[3 * nint + i] = bnw; Lout[4 * nint + i] = bn; Lout[5 * nint + i] = bc;
          Lout[6 * nint + i] = be;
        }
      }
    }
    /* copy beta into gamma, then reset beta (Algorithm 1, end of z loop) */
    memcpy(gamma, beta, sizeof(double) * 8 * M * M);
    for (int d = 0; d < 8; ++d)
      for (int k = 0; k < M * M; ++k) beta[d * M * M + k] = d == C ? 1.0 : 0.0;
  }
#undef B
#undef G
  free(beta); free(gamma);
  return ORC_OK;
fail:
  free(beta); free(gamma);
  return ORC_ERR;
}

/* ------------------------------------------------------- surrogates ---- */

/* Legendre polynomials P_0..P_deg at t (three-term recurrence). */
static void legendre(int deg, double t, double *Pv) {
  Pv[0] = 1.0;
  if (deg >= 1) Pv[1] = t;
  for (int n = 1; n < deg; ++n) Pv[n + 1] = ((2.0 * n + 1.0) * t * Pv[n] - n * Pv[n - 1]) / (n + 1.0);
}

/* Tensor-product surrogate value at logical point (x,y,z):
 *   f(p) = sum_{ijk} c[(i*(dy+1)+j)*(dz+1)+k] P_i(2hx-1) P_j(2hy-1) P_k(2hz-1)
 * with h = 1/N.  The space is the paper's P_{dgx,dgy,dgz} of Sec. 4.1 written
 * in a Legendre basis of each coordinate (same space as the monomials
 * (hx)^i (hy)^j (hz)^k). */
double orc_surrogate_eval(int N, const int *deg, const double *coef, double x, double y, double z) {
  double px[16], py[16], pz[16], h = 1.0 / N;
  legendre(deg[0], 2.0 * h * x - 1.0, px);
  legendre(deg[1], 2.0 * h * y - 1.0, py);
  legendre(deg[2], 2.0 * h * z - 1.0, pz);
  double f = 0.0;
  for (int i = 0; i <= deg[0]; ++i)
    for (int j = 0; j <= deg[1]; ++j)
      for (int k = 0; k <= deg[2]; ++k)
        f += coef[(i * (deg[1] + 1) + j) * (deg[2] + 1) + k] * px[i] * py[j] * pz[k];
  return f;
}

/* Design matrix rows of the same basis at a list of points (for the LSQ). */
int orc_basis_rows(int N, const int *deg, long npts, const double *xyz, double *V) {
  long M = (long)(deg[0] + 1) * (deg[1] + 1) * (deg[2] + 1);
  double px[16], py[16], pz[16], h = 1.0 / N;
  for (long r = 0; r < npts; ++r) {
    legendre(deg[0], 2.0 * h * xyz[3 * r] - 1.0, px);
    legendre(deg[1], 2.0 * h * xyz[3 * r + 1] - 1.0, py);
    legendre(deg[2], 2.0 * h * xyz[3 * r + 2] - 1.0, pz);
    for (int i = 0; i <= deg[0]; ++i)
      for (int j = 0; j <= deg[1]; ++j)
        for (int k = 0; k <= deg[2]; ++k)
          V[r * M + (i * (deg[1] + 1) + j) * (deg[2] + 1) + k] = px[i] * py[j] * pz[k];
  }
  return ORC_OK;
}

/* Sample set S_d of Sec. 4.1: interior points p with
 * (p - (1 - d)) mod stride == 0 componentwise and, for d != c, p + d interior.
 * d is given as a direction index (0..6 for D_l, 7 for c).  Writes the
 * interior numbers of the samples; returns the count. */
long orc_sample_set(int N, int d, int stride, long *out) {
  long i = 0, n = 0;
  for (int z = 1; z <= N - 1; ++z)
    for (int y = 1; y <= N - 1 - z; ++y)
      for (int x = 1; x <= N - 1 - z - y; ++x, ++i) {
        int p[3] = {x, y, z}, ok = 1;
        for (int c = 0; c < 3; ++c) {
          int r = (p[c] - (1 - DIR[d][c])) % stride;
          if (r != 0) ok = 0;
        }
        if (d != 7 && !orc_in_interior(N, x + DIR[d][0], y + DIR[d][1], z + DIR[d][2])) ok = 0;
        if (ok) { if (out) out[n] = i; ++n; }
      }
  return n;
}

/* Evaluate all eight surrogates (L_d for d in D_l, then 1/D) at every
 * interior point; V2 convention: L^p_d = 0 where p+d is not interior
 * (Algorithm 2, lines marked V2). coefs: 8 blocks of M coefficients. */
int orc_eval_all(int N, const int *deg, const double *coefs, double *Lout /* [d*nint+i] */, double *Dinv) {
  long M = (long)(deg[0] + 1) * (deg[1] + 1) * (deg[2] + 1);
  long i = 0, nint = 0;
  for (int z = 1; z <= N - 1; ++z)
    for (int y = 1; y <= N - 1 - z; ++y) nint += (N - 1 - z - y > 0) ? N - 1 - z - y : 0;
  for (int z = 1; z <= N - 1; ++z)
    for (int y = 1; y <= N - 1 - z; ++y)
      for (int x = 1; x <= N - 1 - z - y; ++x, ++i) {
        for (int d = 0; d < 7; ++d)
          Lout[(long)d * nint + i] = orc_in_interior(N, x + DIR[d][0], y + DIR[d][1], z + DIR[d][2])
                                         ? orc_surrogate_eval(N, deg, coefs + d * M, x, y, z)
                                         : 0.0;
        Dinv[i] = orc_surrogate_eval(N, deg, coefs + 7 * M, x, y, z);
      }
  return ORC_OK;
}

/* --------------------------------------------------------- smoother ---- */

/* One or more applications of  x <- x + (L D L^T)^{-1} (b - A x)  on the
 * interior (Algorithm 2, Sec. 4.1; the smoother of Sec. 2.1 with
 * C = L D L^T).  The factor is given per interior point: L[d*nint+i] for
 * d in D_l (already zero where p+d is not interior, the V2 rule) and the
 * inverse pivot Dinv[i].  Forward pass in lexicographic order:
 *   w^p = b^p - sum_{d in D} A^p_d x^{p+d} - sum_{d in D_l} L^p_d w^{p+d};
 * backward pass in reverse order:
 *   w^p = Dinv^p w^p - sum_{d in D_l} L^{p-d}_d w^{p-d};  x^p += w^p.
 * x is the full grid (boundary entries are Dirichlet data and stay fixed);
 * b is the full grid (boundary entries ignored).  rnorm[k] (if non-NULL)
 * receives ||b - A x||_2 over interior rows before sweep k. */
int orc_smooth(int N, const long *rowptr, const long *col, const double *val,
               const double *L, const double *Dinv, double *x, const double *b, int sweeps,
               double *rnorm) {
  long nn = orc_num_nodes(N);
  long *intid = (long *)malloc(sizeof(long) * nn);
  long nint = orc_interior_ids(N, intid);
  long *pts = (long *)malloc(sizeof(long) * nint);
  double *w = (double *)malloc(sizeof(double) * nint);
  int *xyz = (int *)malloc(sizeof(int) * 3 * nn);
  long *rt = row_table(N);
  if (!intid || !pts || !w || !xyz || !rt) {
    free(intid); free(pts); free(w); free(xyz); free(rt);
    return ORC_ERR;
  }
  orc_coords(N, xyz);
  for (long k = 0; k < nn; ++k)
    if (intid[k] >= 0) pts[intid[k]] = k;
  for (int sw = 0; sw < sweeps; ++sw) {
    double rr = 0.0;
    for (long i = 0; i < nint; ++i) {
      long g = pts[i];
      double r = b[g];
      for (long m = rowptr[g]; m < rowptr[g + 1]; ++m) r -= val[m] * x[col[m]];
      rr += r * r;
      int px = xyz[3 * g], py = xyz[3 * g + 1], pz = xyz[3 * g + 2];
      for (int d = 0; d < 7; ++d) {
        int qx = px + DIR[d][0], qy = py + DIR[d][1], qz = pz + DIR[d][2];
        if (orc_in_interior(N, qx, qy, qz)) r -= L[(long)d * nint + i] * w[intid[IDX(rt, N, qx, qy, qz)]];
      }
      w[i] = r;
    }
    if (rnorm) rnorm[sw] = sqrt(rr);
    for (long i = nint - 1; i >= 0; --i) {
      long g = pts[i];
      double v = Dinv[i] * w[i];
      int px = xyz[3 * g], py = xyz[3 * g + 1], pz = xyz[3 * g + 2];
      for (int d = 0; d < 7; ++d) {
        int qx = px - DIR[d][0], qy = py - DIR[d][1], qz = pz - DIR[d][2];
        if (orc_in_interior(N, qx, qy, qz)) {
          long j = intid[IDX(rt, N, qx, qy, qz)];
          v -= L[(long)d * nint + j] * w[j];
        }
      }
      w[i] = v;
      x[g] += v;
    }
  }
  free(intid); free(pts); free(w); free(xyz); free(rt);
  return ORC_OK;
}

/* r = b - A x on interior rows (full-grid vectors; r's boundary entries are
 * set to 0).  Returns ||r||_2. */
double orc_residual(int N, const long *rowptr, const long *col, const double *val,
                    const double *x, const double *b, double *r) {
  double rr = 0.0;
  long k = 0;
  for (int z = 0; z <= N; ++z)
    for (int y = 0; y <= N - z; ++y)
      for (int xx = 0; xx <= N - z - y; ++xx, ++k) {
        if (!orc_in_interior(N, xx, y, z)) { if (r) r[k] = 0.0; continue; }
        double v = b[k];
        for (long m = rowptr[k]; m < rowptr[k + 1]; ++m) v -= val[m] * x[col[m]];
        if (r) r[k] = v;
        rr += v * v;
      }
  return sqrt(rr);
}

/* y = A_tt u on interior points only (boundary treated as zero), interior
 * numbering.  Helper for the Krylov solver below. */
static void matvec_int(long nint, const long *pts, const long *intid, const long *rowptr, const long *col,
                       const double *val, const double *u, double *y) {
  for (long i = 0; i < nint; ++i) {
    long g = pts[i];
    double v = 0.0;
    for (long m = rowptr[g]; m < rowptr[g + 1]; ++m)
      if (intid[col[m]] >= 0) v += val[m] * u[intid[col[m]]];
    y[i] = v;
  }
}

/* Preconditioned conjugate gradients on the interior system
 * A_tt u_t = b_t - A_tG u_G (Dirichlet data from the boundary of x), with
 * the preconditioner C = L D L^T applied by one smoother application from a
 * zero start (Sec. 4.2, "ILU as a preconditioner within a CG method").
 * Stops when ||b - A x||_2 <= rtol ||b_t||_2.  x is updated in place.
 * Returns the iteration count, or -1 on failure / no convergence. */
int orc_pcg(int N, const long *rowptr, const long *col, const double *val, const double *L,
            const double *Dinv, double *x, const double *b, double rtol, int maxit, double *relres) {
  long nn = orc_num_nodes(N);
  long *intid = (long *)malloc(sizeof(long) * nn);
  long nint = orc_interior_ids(N, intid);
  long *pts = (long *)malloc(sizeof(long) * nint);
  double *r = (double *)malloc(sizeof(double) * nint), *z = (double *)malloc(sizeof(double) * nint);
  double *p = (double *)malloc(sizeof(double) * nint), *q = (double *)malloc(sizeof(double) * nint);
  double *fz = (double *)calloc(nn, sizeof(double)), *fr = (double *)calloc(nn, sizeof(double));
  int it = -1;
  if (!intid || !pts || !r || !z || !p || !q || !fz || !fr) goto done;
  for (long k = 0; k < nn; ++k)
    if (intid[k] >= 0) pts[intid[k]] = k;
  double bn = 0.0;
  for (long i = 0; i < nint; ++i) bn += b[pts[i]] * b[pts[i]];
  bn = sqrt(bn);
  double *full_r = (double *)malloc(sizeof(double) * nn);
  if (!full_r) goto done;
  orc_residual(N, rowptr, col, val, x, b, full_r);
  for (long i = 0; i < nint; ++i) r[i] = full_r[pts[i]];
  free(full_r);
  double rz = 0.0;
  for (it = 0; it <= maxit; ++it) {
    double rn = 0.0;
    for (long i = 0; i < nint; ++i) rn += r[i] * r[i];
    rn = sqrt(rn);
    if (relres) *relres = rn / bn;
    if (rn <= rtol * bn) break;
    if (it == maxit) { it = -1; break; }
    /* z = C^{-1} r: one smoother application with zero start and zero boundary */
    for (long k = 0; k < nn; ++k) { fz[k] = 0.0; fr[k] = 0.0; }
    for (long i = 0; i < nint; ++i) fr[pts[i]] = r[i];
    orc_smooth(N, rowptr, col, val, L, Dinv, fz, fr, 1, NULL);
    for (long i = 0; i < nint; ++i) z[i] = fz[pts[i]];
    double rz_new = 0.0;
    for (long i = 0; i < nint; ++i) rz_new += r[i] * z[i];
    if (it == 0) for (long i = 0; i < nint; ++i) p[i] = z[i];
    else for (long i = 0; i < nint; ++i) p[i] = z[i] + (rz_new / rz) * p[i];
    rz = rz_new;
    matvec_int(nint, pts, intid, rowptr, col, val, p, q);
    double pq = 0.0;
    for (long i = 0; i < nint; ++i) pq += p[i] * q[i];
    double alpha = rz / pq;
    for (long i = 0; i < nint; ++i) { x[pts[i]] += alpha * p[i]; r[i] -= alpha * q[i]; }
  }
done:
  free(intid); free(pts); free(r); free(z); free(p); free(q); free(fz); free(fr);
  return it;
}
