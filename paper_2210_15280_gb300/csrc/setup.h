// setup.h -- host-side (FP64) set-up of one macro-tetrahedron: geometry,
// operator stencils, the streaming ILU(0) factorisation, the surrogate fit and
// the per-row evaluation tables the sweep kernels read.
#pragma once
#include <string>
#include <vector>

#include "../../include/ilu.h"
#include "grid.h"

namespace ilu {

struct HostTet {
  int L = 0, N = 0;
  double h = 0;
  double P[4][3] = {};
  ilu_coeff coeff = {};
  int deg[3] = {0, 0, 0};
  int M = 1;            // (dgx+1)(dgy+1)(dgz+1)
  int LH = 5;           // sampling level
  double ridge = 1e-6;  // relative Tikhonov weight
  int factor = 0;       // ilu_factor: ILU(0) (Alg. 1) or symmetric Gauss-Seidel
  int boundary = 0;     // ilu_boundary: V2, or V1 with the cell-boundary factors stored
  std::vector<int> bnd_rowoff;  // V1: first record of each interior row (row_id order), then the total
  std::vector<double> bndL;     // V1: 8 values per cell-boundary point (L^p_d, d in D_l, then 1/D^p), lexicographic
  bool const_kappa = true;
  double Kunit[6][4][4] = {};  // unit-coefficient element matrices of the six micro-tet classes
  int off[6][4][3] = {};       // their vertex offsets
  double A15[15] = {};         // constant-coefficient stencil (includes kappa = c0)
  double W[15][15] = {};       // variable-coefficient edge-star weights (row 7 unused)
  double Wstar[kStarPairs] = {};  // W on the fixed pattern, in star_d/star_q order
  std::vector<double> kappa;   // kappa at every grid point (variable coefficient only)
  std::vector<double> coefs;   // 8 x M surrogate coefficients (Legendre tensor basis)
  bool keep_exact = false;
  std::vector<double> exactL;  // 7 x nint, Alg. 1 factors (kept for small levels)
  std::vector<double> exactD;  // nint
  int dx = 0;                  // x-degree = row polynomial degree
  int rstride = 0;             // padded coefficients per function in the row tables
  std::vector<double> tabF64, tabB64;  // rows x 7 x rstride, rows x 8 x rstride
  std::vector<float> tabF32, tabB32;   // rows x 4 pairs x rstride x 2 (see build_row_tables)
};

// Full set-up.  Returns ILU_OK or an error with a message in err.
ilu_status host_setup(HostTet &t, const double P[12], int level, const ilu_coeff *coeff, const int deg[3],
                      int sample_level, double ridge, std::string &err);
// (Re)build the row tables from t.coefs.
void build_row_tables(HostTet &t);
// Constant 15-point stencil of a tet with kappa = 1 at level 2 (the values at
// level L are these times 2^(2-L)).  False (with err) for a degenerate tet.
bool unit_stencil(const double P[12], double A[15], std::string &err);
// Stencil of the full operator at a grid point (15 directions).
void host_stencil(const HostTet &t, int x, int y, int z, double A[15]);
// Evaluate the eight surrogates from the FP64 row tables (V2-masked L).
void host_eval_tables(const HostTet &t, int x, int y, int z, double out[8]);
// Direct evaluation of surrogate f (0..7) from the 3-D coefficients.
double host_eval_coefs(const HostTet &t, int f, double x, double y, double z);
// Physical coordinates of a logical point.
void host_phys(const HostTet &t, double x, double y, double z, double X[3]);
double host_kappa(const ilu_coeff &c, const double X[3]);

}  // namespace ilu
