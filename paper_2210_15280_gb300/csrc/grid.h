// grid.h -- logical grid of one refined macro-tetrahedron, shared by host and
// device code of the library.
//
// Sec. 2.1 of arXiv 2210.15280: points (x,y,z) with x,y,z >= 0 and
// x+y+z <= N (N = 2^L), interior points with x,y,z >= 1 and x+y+z <= N-1,
// lexicographic order with z slowest and x fastest.  Stencil directions are
// numbered in the order of the paper's set D:
//   0 w  1 s  2 se  3 bnw  4 bn  5 bc  6 be  7 c  8 e  9 n  10 nw  11 tse
//   12 ts 13 tc 14 tw
// The first seven form D_l (the lexicographically lower neighbours); direction
// 8+k is the negative of direction k.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define ILU_HD __host__ __device__ __forceinline__
#define ILU_HDC __host__ __device__ constexpr
#else
#define ILU_HD inline
#define ILU_HDC constexpr
#endif

namespace ilu {

constexpr int kNumDirs = 15;
constexpr int kNumLower = 7;
constexpr int kCentre = 7;

ILU_HD int dir_dx(int d) {
  switch (d) {
    case 0: return -1; case 1: return 0; case 2: return 1; case 3: return -1; case 4: return 0;
    case 5: return 0; case 6: return 1; case 7: return 0; case 8: return 1; case 9: return 0;
    case 10: return -1; case 11: return 1; case 12: return 0; case 13: return 0; default: return -1;
  }
}
ILU_HD int dir_dy(int d) {
  switch (d) {
    case 0: return 0; case 1: return -1; case 2: return -1; case 3: return 1; case 4: return 1;
    case 5: return 0; case 6: return 0; case 7: return 0; case 8: return 0; case 9: return 1;
    case 10: return 1; case 11: return -1; case 12: return -1; case 13: return 0; default: return 0;
  }
}
ILU_HD int dir_dz(int d) {
  switch (d) {
    case 0: return 0; case 1: return 0; case 2: return 0; case 3: return -1; case 4: return -1;
    case 5: return -1; case 6: return -1; case 7: return 0; case 8: return 0; case 9: return 0;
    case 10: return 0; case 11: return 1; case 12: return 1; case 13: return 1; default: return 1;
  }
}
// Hyperplane weight l(d) = dx + 2 dy + 3 dz.  Every d in D_l has l(d) <= -1,
// so points with equal x + 2y + 3z never depend on one another in the
// forward substitution (and symmetrically in the backward one).
ILU_HD int dir_level(int d) { return dir_dx(d) + 2 * dir_dy(d) + 3 * dir_dz(d); }

ILU_HD int64_t tet_number(int64_t m) { return m * (m + 1) * (m + 2) / 6; }

// number of points of G
ILU_HD int64_t grid_nodes(int N) { return tet_number(N + 1); }
// number of interior points
ILU_HD int64_t grid_interior(int N) { return N >= 4 ? tet_number(N - 3) : 0; }
// index of the first point of layer z
ILU_HD int64_t layer_start(int N, int z) { return tet_number(N + 1) - tet_number(N + 1 - z); }
// offset of row y inside layer z (rows have N-z-y+1 points)
ILU_HD int64_t row_offset(int N, int z, int y) {
  const int64_t K = N - z;
  return (int64_t)y * (K + 1) - (int64_t)y * (y - 1) / 2;
}
ILU_HD int64_t grid_index(int N, int x, int y, int z) { return layer_start(N, z) + row_offset(N, z, y) + x; }

ILU_HD bool in_grid(int N, int x, int y, int z) { return x >= 0 && y >= 0 && z >= 0 && x + y + z <= N; }
ILU_HD bool in_interior(int N, int x, int y, int z) { return x >= 1 && y >= 1 && z >= 1 && x + y + z <= N - 1; }

// Interior rows: (y,z) with y,z >= 1 and y+z <= N-2, numbered z-major.
ILU_HD int64_t num_rows(int N) { return N >= 4 ? (int64_t)(N - 3) * (N - 2) / 2 : 0; }
ILU_HD int64_t row_id(int N, int y, int z) {
  return (int64_t)(z - 1) * (N - 2) - (int64_t)(z - 1) * z / 2 + (y - 1);
}
// interior x-range of row (y,z) is [1, N-1-y-z]; its centre
ILU_HD int row_len(int N, int y, int z) { return N - 1 - y - z; }

// ---- 32-bit forms for the kernels (every grid index fits for N <= 1024,
// level 10).  Grid index of (0, y, z); row id.
ILU_HD int row_start32(int N, int y, int z) {
  const int a = N + 1, b = N + 1 - z;
  return (a * (a + 1) * (a + 2) - b * (b + 1) * (b + 2)) / 6 + y * (N - z + 1) - y * (y - 1) / 2;
}
ILU_HD int row_id32(int N, int y, int z) { return (z - 1) * (N - 2) - (z - 1) * z / 2 + (y - 1); }
// The grid indices of (0, .) of the seven rows a stencil at (x, y, z) touches,
// from r0 = row_start32(N, y, z): layer z' holds (N - z' + 1)(N - z' + 2) / 2
// points, row (y, z) N - z - y + 1.
struct StencilRows {
  int r0, rs, rn, rb, rbn, rt, rts;  // (y,z) (y-1,z) (y+1,z) (y,z-1) (y+1,z-1) (y,z+1) (y-1,z+1)
};
ILU_HD StencilRows stencil_rows(int N, int y, int z) {
  StencilRows R;
  const int m = N - z - y;  // row (y, z) has m + 1 points
  R.r0 = row_start32(N, y, z);
  R.rs = R.r0 - (m + 2);
  R.rn = R.r0 + (m + 1);
  R.rb = R.r0 - (N - z + 2) * (N - z + 3) / 2 + y;
  R.rbn = R.rb + m + 2;
  R.rt = R.r0 + (N - z + 1) * (N - z + 2) / 2 - y;
  R.rts = R.rt - (m + 1);
  return R;
}

// ---- residual chunks: the interior points in lexicographic order (x fastest,
// then y, then z), cut into runs of 32; a chunk is the first point of its run,
// x | y << 10 | z << 20.  Lane `lane` of a warp takes the run's point number
// `lane`: false past the last interior point.  All 32 lanes must call it
// together: the rows are stepped through in a warp-uniform loop, so the warp
// leaves it converged (a loop that each lane left on its own would leave the
// lanes to run the stencil arithmetic that follows in separate groups).
#if defined(__CUDACC__)
__device__ __forceinline__ bool chunk_point(int N, int ch, int lane, int &x, int &y, int &z) {
  x = (ch & 1023) + lane;
  y = (ch >> 10) & 1023;
  z = ch >> 20;
  bool ok = true;
  int n = N - 1 - y - z;
  bool more = x > n;
  while (__any_sync(0xffffffffu, more)) {  // the run continues in the next rows (a few at most)
    if (more) {
      x -= n;
      if (++y > N - 2 - z) {
        y = 1;
        if (++z > N - 3) ok = false;
      }
      n = N - 1 - y - z;
      more = ok && x > n;
    }
  }
  return ok;
}
#endif

// ---- boundary variant V1: the interior points on the cell boundary (a
// neighbour in D outside the interior) keep their exact factors.  Rows with
// y = 1 or z = 1 lie wholly on it; every other row has its first (x = 1) and
// last (x + y + z = N - 1) point on it.  Records are numbered in
// lexicographic order; off[row_id] is the first record of a row.
ILU_HD bool on_cell_boundary(int N, int x, int y, int z) { return x == 1 || y == 1 || z == 1 || x + y + z == N - 1; }
ILU_HD int bnd_row_count(int N, int y, int z) {
  const int n = row_len(N, y, z);
  return (y == 1 || z == 1) ? n : (n < 2 ? n : 2);
}
// record of a cell-boundary point (x, y, z), given the row offsets
ILU_HD int bnd_record(const int *off, int N, int x, int y, int z) {
  const int o = off[row_id(N, y, z)];
  return (y == 1 || z == 1) ? o + x - 1 : o + (x == 1 ? 0 : 1);
}

// ---- bands: the FP32 sweeps give each lane of a warp one row.  Band k of
// layer z holds the 32 rows y = band_Y(z,k) + j, j = 0..31 (rows outside
// [1, N-2-z] are idle lanes).  The bands slant by one row per layer, so that
// band k of layer z depends only on bands k-1 and k of layers z and z-1 in
// the forward substitution (and on k, k+1 of z, z+1 in the backward one).
// At step s lane j works on x = s - 2j: all lanes of a band are on the same
// hyperplane x + 2y + 3z = s + band_level0(z,k).
ILU_HD int band_kmax(int N) { return (N - 3) >> 5; }
ILU_HD int band_kmin(int z) { return z >> 5; }
ILU_HD int band_Y(int z, int k) { return 32 * k - z + 1; }
ILU_HD int band_level0(int z, int k) { return 2 * band_Y(z, k) + 3 * z; }
// first and last step with an interior point
ILU_HD int band_slo(int z, int k) {
  const int Y = band_Y(z, k);
  return 1 + 2 * (Y >= 1 ? 0 : 1 - Y);
}
ILU_HD int band_shi(int N, int z, int k) {
  const int Y = band_Y(z, k);
  int jh = N - 2 - z - Y;
  if (jh > 31) jh = 31;
  return N - 1 - Y - z + jh;
}
ILU_HD bool band_exists(int N, int z, int k) { return z >= 1 && z <= N - 3 && k >= band_kmin(z) && k <= band_kmax(N); }

// Edge-star pattern of the variable-coefficient stencil.  With element values
// kappa_T = mean of the vertex values, A^p_d = sum_q W[d][q] kappa(p+q), where
// q runs over the neighbours that share a micro-tetrahedron with the edge
// (p, p+d): 8 of them for w se bn bc e nw ts tc, 6 for the others.  The
// pattern is fixed by the refinement (100 pairs); the set-up checks that every
// nonzero weight it computes lies on it.
constexpr int kStarPairs = 100;
ILU_HDC int star_d(int e) {
  constexpr unsigned char t[kStarPairs] = {
      0,  0,  0,  0,  0,  0,  0,  0,  1,  1,  1,  1,  1,  1,  2,  2,  2,  2,  2,  2,  2,  2,  3,  3,  3,
      3,  3,  3,  4,  4,  4,  4,  4,  4,  4,  4,  5,  5,  5,  5,  5,  5,  5,  5,  6,  6,  6,  6,  6,  6,
      8,  8,  8,  8,  8,  8,  8,  8,  9,  9,  9,  9,  9,  9,  10, 10, 10, 10, 10, 10, 10, 10, 11, 11, 11,
      11, 11, 11, 12, 12, 12, 12, 12, 12, 12, 12, 13, 13, 13, 13, 13, 13, 13, 13, 14, 14, 14, 14, 14, 14};
  return t[e];
}
ILU_HDC int star_q(int e) {
  constexpr unsigned char t[kStarPairs] = {
      0, 1, 3, 5,  7,  10, 12, 14, 0, 1, 2, 5,  7,  12, 1, 2,  5,  6,  7,  8,  11, 12, 0,  3,  4,
      5, 7, 10, 3, 4, 5,  6,  7,  8, 9, 10, 0, 1,  2,  3, 4,  5,  6,  7,  2,  4,  5,  6,  7,  8,
      2, 4, 6,  7, 8, 9,  11, 13, 4, 7, 8,  9, 10, 13, 0, 3,  4,  7,  9,  10, 13, 14, 2,  7,  8,
      11, 12, 13, 0, 1, 2, 7,  11, 12, 13, 14, 7, 8, 9, 10, 11, 12, 13, 14, 0,  7,  10, 12, 13, 14};
  return t[e];
}

}  // namespace ilu
