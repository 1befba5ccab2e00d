"""Python face of the CPU oracle (oracle.c) plus the least-squares fit.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py; never by the library.  It shares no code with
the library in paper_2210_15280_gb300/.

Parity of the surrogate fit is pinned by tests/test_oracle.py; every function
here names the passage of arXiv 2210.15280 it follows.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

# direction names in the order of the paper's set D (Sec. 2.1)
DIRS = ["w", "s", "se", "bnw", "bn", "bc", "be", "c", "e", "n", "nw", "tse", "ts", "tc", "tw"]
DL = DIRS[:7]
COEFF_KINDS = {"const": 0, "sinprod": 1, "kappa_i": 2}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, plain C99)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", _SO, src, "-lm"])
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
        vp = ctypes.c_void_p
        L.orc_num_nodes.restype = l; L.orc_num_nodes.argtypes = [i]
        L.orc_index.restype = l; L.orc_index.argtypes = [i, i, i, i]
        L.orc_coords.argtypes = [i, vp]
        L.orc_enumerate_tets.restype = l; L.orc_enumerate_tets.argtypes = [i, vp]
        L.orc_phys.argtypes = [vp, i, d, d, d, vp]
        L.orc_kappa.restype = d; L.orc_kappa.argtypes = [i, d, d, i, vp]
        L.orc_element.restype = d; L.orc_element.argtypes = [vp, vp, vp]
        L.orc_assemble.restype = l
        L.orc_assemble.argtypes = [i, vp, i, d, d, i, vp, vp, vp, l]
        L.orc_local_stencil.argtypes = [i, vp, i, d, d, i, i, i, i, vp]
        L.orc_interior_ids.restype = l; L.orc_interior_ids.argtypes = [i, vp]
        L.orc_ilu0.argtypes = [i, vp, vp, vp, vp, vp]
        L.orc_sgs_factors.argtypes = [i, vp, vp, vp, vp, vp]
        L.orc_sgs_sweep.argtypes = [i, vp, vp, vp, vp, vp]
        L.orc_alg1.argtypes = [i, vp, i, d, d, i, vp, vp]
        L.orc_surrogate_eval.restype = d; L.orc_surrogate_eval.argtypes = [i, vp, vp, d, d, d]
        L.orc_basis_rows.argtypes = [i, vp, l, vp, vp]
        L.orc_sample_set.restype = l; L.orc_sample_set.argtypes = [i, i, i, vp]
        L.orc_eval_all.argtypes = [i, vp, vp, vp, vp]
        L.orc_smooth.argtypes = [i, vp, vp, vp, vp, vp, vp, vp, i, vp]
        L.orc_residual.restype = d; L.orc_residual.argtypes = [i, vp, vp, vp, vp, vp, vp]
        L.orc_pcg.argtypes = [i, vp, vp, vp, vp, vp, vp, vp, d, i, vp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ grid ---

def num_nodes(N):
    return lib().orc_num_nodes(N)


def coords(N):
    """(n,3) int array of the logical coordinates of G in lexicographic order."""
    out = np.zeros((num_nodes(N), 3), dtype=np.int32)
    lib().orc_coords(N, _p(out))
    return out


def interior_ids(N):
    ids = np.zeros(num_nodes(N), dtype=np.int64)
    nint = lib().orc_interior_ids(N, _p(ids))
    return ids, nint


def index(N, x, y, z):
    return lib().orc_index(N, x, y, z)


def tets(N):
    n = lib().orc_enumerate_tets(N, None)
    out = np.zeros((n, 4, 3), dtype=np.int32)
    lib().orc_enumerate_tets(N, _p(out))
    return out


def phys(P, N, xyz):
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(12)
    xyz = np.asarray(xyz, dtype=np.float64)
    # the same affine map as orc_phys, vectorised for tests
    out = np.zeros(3)
    lib().orc_phys(_p(P), N, float(xyz[0]), float(xyz[1]), float(xyz[2]), _p(out))
    return out


def element(X, kv):
    X = np.ascontiguousarray(X, dtype=np.float64)
    kv = np.ascontiguousarray(kv, dtype=np.float64)
    K = np.zeros((4, 4))
    vol = lib().orc_element(_p(X), _p(kv), _p(K))
    return K, vol


# ------------------------------------------------------------ assembly ---

class Coeff:
    """kappa: kind in {const, sinprod, kappa_i} with parameters (Sec. 4.2 for kappa_i)."""

    def __init__(self, kind="const", c0=1.0, amp=0.0, ipow=0):
        self.kind, self.c0, self.amp, self.ipow = kind, float(c0), float(amp), int(ipow)

    def args(self):
        return COEFF_KINDS[self.kind], self.c0, self.amp, self.ipow


def assemble(P, N, coeff=None):
    """Global P1 stiffness matrix on all of G (CSR arrays, sorted columns)."""
    coeff = coeff or Coeff()
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(12)
    nn = num_nodes(N)
    cap = 15 * nn
    rowptr = np.zeros(nn + 1, dtype=np.int64)
    col = np.zeros(cap, dtype=np.int64)
    val = np.zeros(cap)
    nz = lib().orc_assemble(N, _p(P), *coeff.args(), _p(rowptr), _p(col), _p(val), cap)
    if nz < 0:
        raise RuntimeError("oracle assembly failed (row capacity)")
    return rowptr, col[:nz].copy(), val[:nz].copy()


def local_stencil(P, N, p, coeff=None):
    coeff = coeff or Coeff()
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(12)
    st = np.zeros(15)
    rc = lib().orc_local_stencil(N, _p(P), *coeff.args(), int(p[0]), int(p[1]), int(p[2]), _p(st))
    if rc != 0:
        raise RuntimeError("local stencil: coupling outside D")
    return st


def to_scipy(A, N):
    import scipy.sparse as sp
    rowptr, col, val = A
    n = num_nodes(N)
    return sp.csr_matrix((val, col, rowptr), shape=(n, n))


# -------------------------------------------------------------- ILU(0) ---

def ilu0(A, N):
    """Exact ILU(0) of the interior block (IKJ elimination).  Returns
    (L[7, nint], D[nint]) in interior lexicographic order."""
    rowptr, col, val = A
    _, nint = interior_ids(N)
    L = np.zeros((7, nint)); D = np.zeros(nint)
    rc = lib().orc_ilu0(N, _p(rowptr), _p(col), _p(val), _p(L), _p(D))
    if rc != 0:
        raise RuntimeError("oracle ILU(0): non-positive pivot")
    return L, D


def sgs_factors(A, N):
    """Symmetric Gauss-Seidel in the L D L^T form of the smoother:
    (L[7, nint], D[nint]) with L^p_d = A(p, p+d) / A(p+d, p+d), D^p = A(p, p)."""
    rowptr, col, val = A
    _, nint = interior_ids(N)
    L = np.zeros((7, nint)); D = np.zeros(nint)
    if lib().orc_sgs_factors(N, _p(rowptr), _p(col), _p(val), _p(L), _p(D)) != 0:
        raise RuntimeError("oracle SGS factors failed")
    return L, D


def sgs_sweep(A, N, x, b):
    """One textbook symmetric Gauss-Seidel sweep (forward then backward),
    in place on x."""
    rowptr, col, val = A
    assert x.dtype == np.float64 and x.flags.c_contiguous
    bb = np.ascontiguousarray(b, dtype=np.float64)
    if lib().orc_sgs_sweep(N, _p(rowptr), _p(col), _p(val), _p(x), _p(bb)) != 0:
        raise RuntimeError("oracle SGS sweep failed")
    return x


def alg1(P, N, coeff=None):
    """Algorithm 1 (streaming in-place LDL^T).  Returns (L[7, nint], D[nint])."""
    coeff = coeff or Coeff()
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(12)
    _, nint = interior_ids(N)
    L = np.zeros((7, nint)); D = np.zeros(nint)
    rc = lib().orc_alg1(N, _p(P), *coeff.args(), _p(L), _p(D))
    if rc != 0:
        raise RuntimeError("oracle Algorithm 1 failed")
    return L, D


# ----------------------------------------------------------- surrogate ---

def sample_set(N, d, stride):
    """Interior numbers of the sample set S_d (d: 0..6 for D_l, 7 for c)."""
    n = lib().orc_sample_set(N, d, stride, None)
    out = np.zeros(n, dtype=np.int64)
    lib().orc_sample_set(N, d, stride, _p(out))
    return out


def basis_rows(N, deg, pts):
    deg = np.ascontiguousarray(deg, dtype=np.int32)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    M = int(np.prod(np.asarray(deg) + 1))
    V = np.zeros((len(pts), M))
    lib().orc_basis_rows(N, _p(deg), len(pts), _p(pts), _p(V))
    return V


def default_sample_level(L):
    return min(L, 5)


def fit_surrogates(N, L_fac, D_fac, deg, sample_level=None, ridge=1e-6):
    """Least-squares surrogates of Sec. 4.1: for each d in D_l the factor
    entries L^p_d at p in S_d, and 1/D^p_c at p in S_c, are fitted in the
    tensor space P_{dgx,dgy,dgz} of the h-scaled coordinates.  The space on a
    tetrahedron is numerically rank deficient, so the fit minimises
    ||V c - t||^2 + (ridge * sqrt(|S_d|))^2 ||c||^2 in the Legendre tensor
    basis (ridge = 0 gives the plain least-squares problem).
    Returns coefficients of shape (8, M)."""
    deg = [int(v) for v in deg]
    level = int(round(np.log2(N)))
    LH = default_sample_level(level) if sample_level is None else sample_level
    stride = max(2 ** (level - LH), 1)
    xyz = interior_coords(N)
    M = int(np.prod(np.asarray(deg) + 1))
    coefs = np.zeros((8, M))
    for d in range(8):
        S = sample_set(N, d, stride)
        t = L_fac[d][S] if d < 7 else 1.0 / D_fac[S]
        V = basis_rows(N, deg, xyz[S].astype(np.float64))
        lam = ridge * np.sqrt(len(S))
        Va = np.vstack([V, lam * np.eye(M)]) if ridge > 0 else V
        ta = np.concatenate([t, np.zeros(M)]) if ridge > 0 else t
        coefs[d] = np.linalg.lstsq(Va, ta, rcond=None)[0]
    return coefs


def interior_coords(N):
    c = coords(N)
    ids, nint = interior_ids(N)
    out = np.zeros((nint, 3), dtype=np.int32)
    out[ids[ids >= 0]] = c[ids >= 0]
    return out


def surrogate_eval(N, deg, coef, p):
    deg = np.ascontiguousarray(deg, dtype=np.int32)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    return lib().orc_surrogate_eval(N, _p(deg), _p(coef), float(p[0]), float(p[1]), float(p[2]))


def eval_surrogates(N, deg, coefs):
    """All eight surrogates at every interior point, V2-masked:
    returns (L[7, nint], Dinv[nint])."""
    deg = np.ascontiguousarray(deg, dtype=np.int32)
    coefs = np.ascontiguousarray(coefs, dtype=np.float64)
    _, nint = interior_ids(N)
    L = np.zeros((7, nint)); Dinv = np.zeros(nint)
    lib().orc_eval_all(N, _p(deg), _p(coefs), _p(L), _p(Dinv))
    return L, Dinv


def cell_boundary_mask(N):
    """Interior points on the cell boundary, in interior order: those with a
    neighbour in D outside the interior, i.e. x = 1, y = 1, z = 1 or
    x + y + z = N - 1 (the points whose factors variant V1 stores, Sec. 4.1)."""
    c = interior_coords(N)
    return (c[:, 0] == 1) | (c[:, 1] == 1) | (c[:, 2] == 1) | (c.sum(axis=1) == N - 1)


def v1_factors(N, L_sur, Dinv_sur, L_exact, D_exact):
    """Boundary variant V1 (Sec. 4.1, Alg. 1): at the cell-boundary points the
    exact ILU(0) factors stored by the factorisation replace the surrogates,
    elsewhere the surrogates stay.  Both stored fields are used: L^p_d
    (d in D_l) and the multiplicative inverse 1/D^p of the centre, which
    Alg. 1 stores for V1 next to the L entries and which the V1 description
    of Sec. 4.1 says the substitutions use.  Returns (L, Dinv); Alg. 2 applied
    with these fields is the V1 smoother."""
    m = cell_boundary_mask(N)
    L = np.array(L_sur, dtype=np.float64, copy=True)
    L[:, m] = L_exact[:, m]
    Dinv = np.array(Dinv_sur, dtype=np.float64, copy=True)
    Dinv[m] = 1.0 / np.asarray(D_exact, dtype=np.float64)[m]
    return L, Dinv


# direction vectors of D in the order of DIRS (Sec. 2.1, with b = z-1, t = z+1)
DVEC = [(-1, 0, 0), (0, -1, 0), (1, -1, 0), (-1, 1, -1), (0, 1, -1), (0, 0, -1), (1, 0, -1), (0, 0, 0),
        (1, 0, 0), (0, 1, 0), (-1, 1, 0), (1, -1, 1), (0, -1, 1), (0, 0, 1), (-1, 0, 1)]


def _interior(N, q):
    return q[0] >= 1 and q[1] >= 1 and q[2] >= 1 and q[0] + q[1] + q[2] <= N - 1


def local_residual(P, N, coeff, x_at, b_at, p):
    """r_p = b_p - sum_{d in D} A^p_d x^{p+d} at one interior point p
    (Alg. 2, all 15 directions, boundary x = Dirichlet data), with the
    element-assembled stencil of p; x_at, b_at map a point to its value."""
    A = local_stencil(P, N, p, coeff)
    r = b_at(p)
    for d, v in enumerate(DVEC):
        r -= A[d] * x_at((p[0] + v[0], p[1] + v[1], p[2] + v[2]))
    return r


def ldlt_apply_at(N, deg, coefs, w_at, p, cache=None):
    """(L~ D~ L~^T w)_p at one interior point p for the surrogate factors
    with the V2 rule (Sec. 3, Alg. 2): L~ unit lower triangular with
    L~_{q, q+d} = L~^q_d (d in D_l, zero where q+d is not interior),
    D~ = diag(1 / D~^-1), every value from the surrogate polynomials (direct
    tensor evaluation).  w_at maps an interior point to w there.  The smoother
    solves C~ w = r, so at every p this equals r_p."""
    cache = {} if cache is None else cache

    def vals(q):  # L~^q_d (d in D_l) and D~^-1(q), unmasked
        v = cache.get(q)
        if v is None:
            v = [surrogate_eval(N, deg, coefs[f], q) for f in range(8)]
            cache[q] = v
        return v

    def lt_w(q):  # (L~^T w)_q = w_q + sum_{d in D_l, q-d interior} L~^{q-d}_d w_{q-d}
        s = w_at(q)
        for d in range(7):
            m = (q[0] - DVEC[d][0], q[1] - DVEC[d][1], q[2] - DVEC[d][2])
            if _interior(N, m):
                s += vals(m)[d] * w_at(m)
        return s

    out = lt_w(p) / vals(p)[7]
    for d in range(7):
        q = (p[0] + DVEC[d][0], p[1] + DVEC[d][1], p[2] + DVEC[d][2])
        if _interior(N, q):
            out += vals(p)[d] * lt_w(q) / vals(q)[7]
    return out


# ------------------------------------------------------------ smoother ---

def smooth(A, N, L, Dinv, x, b, sweeps=1, want_norms=False):
    """Algorithm 2 with the V2 boundary rule: `sweeps` applications of
    x <- x + (L D L^T)^{-1}(b - A x).  x is modified in place (and returned)."""
    rowptr, col, val = A
    L = np.ascontiguousarray(L, dtype=np.float64)
    Dinv = np.ascontiguousarray(Dinv, dtype=np.float64)
    assert x.dtype == np.float64 and x.flags.c_contiguous
    b = np.ascontiguousarray(b, dtype=np.float64)
    norms = np.zeros(max(sweeps, 1))
    lib().orc_smooth(N, _p(rowptr), _p(col), _p(val), _p(L), _p(Dinv), _p(x), _p(b), sweeps,
                     _p(norms) if want_norms else None)
    return (x, norms[:sweeps]) if want_norms else x


def residual(A, N, x, b):
    rowptr, col, val = A
    r = np.zeros(num_nodes(N))
    x = np.ascontiguousarray(x, dtype=np.float64); b = np.ascontiguousarray(b, dtype=np.float64)
    nrm = lib().orc_residual(N, _p(rowptr), _p(col), _p(val), _p(x), _p(b), _p(r))
    return r, nrm


def interior_norm(N, v):
    ids, _ = interior_ids(N)
    return float(np.linalg.norm(v[ids >= 0]))


def richardson(A, N, L, Dinv, x, b, rtol=1e-8, max_iter=100000):
    """Smoothed Richardson iteration x <- x + C^{-1}(b - A x) until the
    relative interior residual is below rtol.  Returns (iters, relres)."""
    bn = interior_norm(N, b)
    for it in range(max_iter + 1):
        _, rn = residual(A, N, x, b)
        if rn <= rtol * bn:
            return it, rn / bn
        if it == max_iter:
            break
        smooth(A, N, L, Dinv, x, b, 1)
    return -1, rn / bn


def pcg(A, N, L, Dinv, x, b, rtol=1e-8, max_iter=10000):
    """CG preconditioned by the ILU smoother (Sec. 4.2).  Returns (iters, relres)."""
    rowptr, col, val = A
    rel = np.zeros(1)
    it = lib().orc_pcg(N, _p(rowptr), _p(col), _p(val), _p(np.ascontiguousarray(L)),
                       _p(np.ascontiguousarray(Dinv)), _p(x), _p(np.ascontiguousarray(b)), rtol, max_iter,
                       _p(rel))
    return it, float(rel[0])


# ---------------------------------------------------- convenience setup ---

class Problem:
    """Everything the oracle knows about one macro-tetrahedron at one level:
    the assembled matrix, the exact ILU(0) and (optionally) the surrogate fit."""

    def __init__(self, P, level, coeff=None, deg=None, sample_level=None, ridge=1e-6, use_alg1=False,
                 factor="ilu"):
        self.P = np.ascontiguousarray(P, dtype=np.float64).reshape(4, 3)
        self.level, self.N = level, 2 ** level
        self.coeff = coeff or Coeff()
        self.A = assemble(self.P, self.N, self.coeff)
        if factor == "sgs":
            self.L, self.D = sgs_factors(self.A, self.N)
        elif use_alg1:
            self.L, self.D = alg1(self.P, self.N, self.coeff)
        else:
            self.L, self.D = ilu0(self.A, self.N)
        self.deg = None
        if deg is not None:
            self.set_degree(deg, sample_level, ridge)

    def set_degree(self, deg, sample_level=None, ridge=1e-6):
        if np.isscalar(deg):
            deg = [int(deg)] * 3
        self.deg = list(deg)
        self.coefs = fit_surrogates(self.N, self.L, self.D, self.deg, sample_level, ridge)
        self.Ls, self.Dinv_s = eval_surrogates(self.N, self.deg, self.coefs)

    def exact_factors(self):
        return self.L, 1.0 / self.D

    def surrogate_factors(self):
        return self.Ls, self.Dinv_s
