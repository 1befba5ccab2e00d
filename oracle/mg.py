"""Geometric multigrid on one macro-tetrahedron, for the convergence study of
arXiv 2210.15280 (Sec. 4.2 numerical results, Table 2, the height study).

TEST INFRASTRUCTURE ONLY: imported by tests/ and by the CPU leg of bench.py;
never by the library, with which it shares no code.

The hierarchy is the nested family of uniformly refined lattices of levels
coarsest..finest on one macro-tet (Sec. 2.1).  Each level has its own
assembled P1 stiffness matrix and its own smoother factors (exact ILU(0) or
symmetric Gauss-Seidel in L D L^T form), applied by the Algorithm 2 smoother.
Grid transfer is the natural one for nested P1 spaces:
  - prolongation: the coarse piecewise-linear function evaluated at the fine
    nodes, built element by element from barycentric coordinates of the
    coarse micro-tets;
  - restriction: its transpose.
The coarsest problem is solved exactly (the paper runs CG there to
convergence).  The asymptotic convergence factor is the ratio of successive
error norms after a 20-step power iteration on the error propagation
operator from a random initial error (Sec. 4.2).
"""
import functools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import oracle as orc


@functools.lru_cache(maxsize=None)
def prolongation(Nc):
    """Sparse (num_nodes(2 Nc) x num_nodes(Nc)) matrix over the full grids:
    row f holds the values at fine node f of the coarse hat functions.  Every
    fine node lies in some coarse micro-tet T; there the coarse hats are the
    barycentric coordinates of T, evaluated at the fine node (in lattice
    coordinates, where the map of Sec. 2.1 is affine, so barycentric
    coordinates are the same as in physical space)."""
    Nf = 2 * Nc

    def lookup(N):
        tab = -np.ones((N + 1,) * 3, dtype=np.int64)
        c = orc.coords(N)
        tab[c[:, 0], c[:, 1], c[:, 2]] = np.arange(len(c))
        return tab

    tc, tf = lookup(Nc), lookup(Nf)
    T = orc.tets(Nc).astype(np.int64)  # (nt, 4, 3) coarse micro-tets
    rows, cols, vals = [], [], []
    seen = np.zeros(orc.num_nodes(Nf), dtype=bool)
    for t in T:
        M = np.vstack([t.T.astype(np.float64), np.ones(4)])  # columns: (x, y, z, 1) of each vertex
        Minv = np.linalg.inv(M)
        cid = [tc[tuple(v)] for v in t]
        # the fine nodes of T: its vertices (doubled) and its edge midpoints
        cand = [2 * t[i] for i in range(4)] + [t[i] + t[j] for i in range(4) for j in range(i + 1, 4)]
        for f in cand:
            fi = tf[tuple(f)]
            if seen[fi]:
                continue
            seen[fi] = True
            lam = Minv @ np.append(f / 2.0, 1.0)
            for k in range(4):
                if abs(lam[k]) > 1e-14:
                    rows.append(fi); cols.append(cid[k]); vals.append(lam[k])
    assert seen.all()
    return sp.csr_matrix((vals, (rows, cols)), shape=(orc.num_nodes(Nf), orc.num_nodes(Nc)))


class Level:
    def __init__(self, P, level, coeff, smoother, factors=None):
        self.level, self.N = level, 2 ** level
        self.A = orc.assemble(P, self.N, coeff)
        ids, self.nint = orc.interior_ids(self.N)
        self.inner = np.nonzero(ids >= 0)[0]
        if factors is not None:  # given (L[7, nint], D^-1[nint]), e.g. surrogate values
            self.L, self.Dinv = factors
            return
        if smoother == "ilu":
            L, D = orc.ilu0(self.A, self.N)
        elif smoother == "sgs":
            L, D = orc.sgs_factors(self.A, self.N)
        else:
            raise ValueError(smoother)
        self.L, self.Dinv = L, 1.0 / D


class Hierarchy:
    """Levels coarsest..finest of one macro-tet with the given smoother and
    nu_pre = nu_post smoothing steps of the V-cycle.  `factors` (optional)
    maps a level to the (L, D^-1) its smoother uses instead of the exact
    factors, e.g. the values of surrogate polynomials."""

    def __init__(self, P, finest, coarsest=2, coeff=None, smoother="ilu", nu=3, factors=None):
        P = np.ascontiguousarray(P, dtype=np.float64).reshape(4, 3)
        coeff = coeff or orc.Coeff()
        factors = factors or {}
        self.nu, self.coarsest, self.finest = nu, coarsest, finest
        self.lv = {l: Level(P, l, coeff, smoother, factors.get(l)) for l in range(coarsest, finest + 1)}
        # interior-to-interior transfers (the correction vanishes on the boundary)
        self.Pm = {}
        for l in range(coarsest + 1, finest + 1):
            Pf = prolongation(2 ** (l - 1))
            self.Pm[l] = Pf[self.lv[l].inner][:, self.lv[l - 1].inner].tocsr()
        c = self.lv[coarsest]
        Ac = orc.to_scipy(c.A, c.N)[c.inner][:, c.inner].tocsc()
        self.coarse = spla.splu(Ac)

    def vcycle(self, l, x, b):
        """One V-cycle on level l for A x = b (full-grid vectors; the boundary
        entries of x are fixed data, those of b ignored); x in place."""
        lv = self.lv[l]
        if l == self.coarsest:
            r, _ = orc.residual(lv.A, lv.N, x, b)
            x[lv.inner] += self.coarse.solve(r[lv.inner])
            return x
        orc.smooth(lv.A, lv.N, lv.L, lv.Dinv, x, b, self.nu)
        r, _ = orc.residual(lv.A, lv.N, x, b)
        c = self.lv[l - 1]
        bc = np.zeros(orc.num_nodes(c.N))
        bc[c.inner] = self.Pm[l].T @ r[lv.inner]
        xc = np.zeros(orc.num_nodes(c.N))
        self.vcycle(l - 1, xc, bc)
        x[lv.inner] += self.Pm[l] @ xc[c.inner]
        orc.smooth(lv.A, lv.N, lv.L, lv.Dinv, x, b, self.nu)
        return x

    def rate(self, e0, steps=20):
        """Power iteration on the error propagation operator: b = 0, x = e0
        (interior, boundary 0), normalised after every V-cycle.  Returns
        (rho, history) with rho the last ratio of successive error norms."""
        lv = self.lv[self.finest]
        x = np.zeros(orc.num_nodes(lv.N))
        x[lv.inner] = e0
        x /= np.linalg.norm(x)
        b = np.zeros_like(x)
        hist = []
        for _ in range(steps):
            self.vcycle(self.finest, x, b)
            n = np.linalg.norm(x)
            hist.append(n)
            x /= n
        return hist[-1], hist

    def iterations(self, e0, reduction=1e-6, max_iter=500):
        """V-cycles until the error norm (b = 0, x = e0) drops by `reduction`."""
        lv = self.lv[self.finest]
        x = np.zeros(orc.num_nodes(lv.N))
        x[lv.inner] = e0
        n0 = np.linalg.norm(x)
        b = np.zeros_like(x)
        for it in range(1, max_iter + 1):
            self.vcycle(self.finest, x, b)
            if np.linalg.norm(x) <= reduction * n0:
                return it
        return -1
