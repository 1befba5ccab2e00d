"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: counts and
volumes of the refinement, polynomial exactness of P1 finite elements, an
independent dense assembly, the defining identity of ILU(0), the paper's own
Algorithm 1 against textbook IKJ elimination, the scaling remark and the
asymptotic stencil of Sec. 3, dense linear algebra for the smoother, and exact
reproduction of polynomials by the fit.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse.linalg as spla

import seeded_inputs as si


def tet_volume(P):
    P = np.asarray(P)
    return abs(np.linalg.det(P[1:] - P[0])) / 6.0


# ----------------------------------------------------------------- grid ---

@pytest.mark.parametrize("level", [2, 3, 4, 5, 6])
def test_grid_counts(orc, level):
    N = 2 ** level
    assert orc.num_nodes(N) == math.comb(N + 3, 3)
    _, nint = orc.interior_ids(N)
    assert nint == math.comb(N - 1, 3)


def test_lexicographic_order(orc):
    """Sec. 2.1: i < j iff (z, y, x) of i precedes that of j."""
    N = 8
    c = orc.coords(N)
    keys = [(z, y, x) for x, y, z in c]
    assert keys == sorted(keys)
    for k in [0, 7, 100, len(c) - 1]:
        x, y, z = c[k]
        assert orc.index(N, int(x), int(y), int(z)) == k


# ----------------------------------------------------------------- mesh ---

@pytest.mark.parametrize("level", [2, 3, 4])
def test_refinement_count_and_volume(orc, level):
    """Uniform 8-way refinement (Sec. 2.1): 8^L micro-tets of equal volume
    filling the macro-tetrahedron."""
    N = 2 ** level
    P = si.macro_tet(11)
    T = orc.tets(N)
    assert len(T) == N ** 3
    vols = []
    for t in T:
        X = np.array([orc.phys(P, N, v) for v in t])
        vols.append(tet_volume(X))
    vols = np.array(vols)
    assert np.allclose(vols, tet_volume(P) / N ** 3, rtol=1e-12)
    assert abs(vols.sum() - tet_volume(P)) < 1e-13


@pytest.mark.parametrize("level", [2, 3])
def test_refinement_conforming(orc, level):
    """Every micro-face is shared by two micro-tets, except faces on the four
    macro faces x=0, y=0, z=0, x+y+z=N, which belong to one."""
    N = 2 ** level
    faces = {}
    for t in orc.tets(N):
        for f in itertools.combinations(range(4), 3):
            key = tuple(sorted(tuple(int(v) for v in t[i]) for i in f))
            faces[key] = faces.get(key, 0) + 1
    for key, n in faces.items():
        V = np.array(key)
        on_boundary = any(np.all(V[:, c] == 0) for c in range(3)) or np.all(V.sum(1) == N)
        assert n == (1 if on_boundary else 2), key


def test_edges_are_stencil_directions(orc):
    """The edge vectors of the micro-mesh are exactly the 14 non-centre
    directions of the paper's stencil set D (Sec. 2.1)."""
    dirs = {tuple(orc.lib().orc_dir(k, c) for c in range(3)) for k in range(15)}
    edges = set()
    for t in orc.tets(4):
        for i in range(4):
            for j in range(4):
                edges.add(tuple(int(v) for v in t[j] - t[i]))
    assert edges == dirs
    # D_l holds the seven directions pointing to lexicographically lower points
    for k in range(7):
        d = [orc.lib().orc_dir(k, c) for c in range(3)]
        assert (d[2], d[1], d[0]) < (0, 0, 0)
    for k in range(8, 15):
        d = [orc.lib().orc_dir(k, c) for c in range(3)]
        assert (d[2], d[1], d[0]) > (0, 0, 0)
        assert d == [-orc.lib().orc_dir(k - 8, c) for c in range(3)]


# ------------------------------------------------------------- assembly ---

def dense_assembly_numpy(orc, P, N, kappa):
    """Independent dense P1 assembly: gradients from the inverse of the 4x4
    matrix [1 X], element matrices |T| k_T G^T G."""
    c = orc.coords(N)
    idx = {tuple(int(v) for v in p): k for k, p in enumerate(c)}
    n = len(c)
    A = np.zeros((n, n))
    for t in orc.tets(N):
        X = np.array([orc.phys(P, N, v) for v in t])
        M = np.hstack([np.ones((4, 1)), X])
        G = np.linalg.inv(M)[1:]
        vol = abs(np.linalg.det(M)) / 6.0
        kT = np.mean([kappa(x) for x in X])
        K = vol * kT * G.T @ G
        ids = [idx[tuple(int(v) for v in p)] for p in t]
        for a in range(4):
            for b in range(4):
                A[ids[a], ids[b]] += K[a, b]
    return A


@pytest.mark.parametrize("level", [2, 3])
def test_assembly_matches_independent_dense(orc, level):
    N = 2 ** level
    P = si.macro_tet(5)
    A = orc.to_scipy(orc.assemble(P, N), N).toarray()
    B = dense_assembly_numpy(orc, P, N, lambda x: 1.0)
    assert np.abs(A - B).max() < 1e-13 * np.abs(B).max()
    co = orc.Coeff("sinprod", 1.0, 0.5)
    A = orc.to_scipy(orc.assemble(P, N, co), N).toarray()
    kap = lambda X: 1.0 + 0.5 * np.prod(np.sin(2 * np.pi * np.asarray(X)))
    B = dense_assembly_numpy(orc, P, N, kap)
    assert np.abs(A - B).max() < 1e-13 * np.abs(B).max()


def test_assembly_symmetric_zero_rowsum(orc):
    N = 16
    P = si.macro_tet(6)
    S = orc.to_scipy(orc.assemble(P, N, orc.Coeff("sinprod", 1.0, 0.5)), N)
    assert abs(S - S.T).max() < 1e-15
    assert np.abs(S @ np.ones(S.shape[0])).max() < 1e-14


def test_couplings_within_D(orc):
    N = 16
    P = si.macro_tet(7)
    rowptr, col, _ = orc.assemble(P, N)
    c = orc.coords(N)
    dirs = {tuple(orc.lib().orc_dir(k, cc) for cc in range(3)) for k in range(15)}
    for r in range(len(c)):
        for m in range(rowptr[r], rowptr[r + 1]):
            assert tuple(int(v) for v in c[col[m]] - c[r]) in dirs


def test_p1_exactness_linear_and_quadratic(orc):
    """For kappa = 1 and interior rows: A u = 0 for u linear, and for
    u = |X|^2 (Laplace u = 6): (A u)_p = -int phi_p Laplace u = -6 * 24 |T| / 4."""
    N = 16
    P = si.macro_tet(8)
    S = orc.to_scipy(orc.assemble(P, N), N)
    c = orc.coords(N)
    X = np.array([orc.phys(P, N, p) for p in c])
    ids, _ = orc.interior_ids(N)
    inter = ids >= 0
    u1 = 0.3 + X @ np.array([1.0, -2.0, 0.5])
    assert np.abs((S @ u1)[inter]).max() < 1e-13
    u2 = (X ** 2).sum(1)
    Tvol = tet_volume(P) / N ** 3
    assert np.allclose((S @ u2)[inter], -36.0 * Tvol, rtol=1e-11)


def test_vertex_mean_kappa_exact_for_linear_kappa(orc):
    """The quadrature kappa_T = mean of the vertex values is exact for a
    linear coefficient: compare with a 4-point Gauss rule on one element."""
    P = si.macro_tet(9)
    X = np.array([orc.phys(P, 4, v) for v in orc.tets(4)[17]])
    kap = lambda Y: orc.lib().orc_kappa(2, 0.0, 0.0, 1, np.ascontiguousarray(Y).ctypes.data_as(orc.ctypes.c_void_p))
    kv = np.array([kap(x) for x in X])
    K, vol = orc.element(X, kv)
    M = np.hstack([np.ones((4, 1)), X]); G = np.linalg.inv(M)[1:]
    a, b = 0.5854101966249685, 0.1381966011250105  # degree-2 Gauss rule on a tetrahedron
    quad = 0.0
    for k in range(4):
        lam = np.full(4, b); lam[k] = a
        quad += 0.25 * kap(lam @ X)
    assert np.allclose(K, vol * quad * G.T @ G, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("level", [3, 4])
def test_local_stencil_matches_global(orc, level):
    N = 2 ** level
    P = si.macro_tet(10)
    co = orc.Coeff("sinprod", 1.0, 0.5)
    rowptr, col, val = orc.assemble(P, N, co)
    c = orc.coords(N)
    for r in range(len(c)):
        st = orc.local_stencil(P, N, c[r], co)
        for m in range(rowptr[r], rowptr[r + 1]):
            d = tuple(int(v) for v in c[col[m]] - c[r])
            k = [tuple(orc.lib().orc_dir(kk, cc) for cc in range(3)) for kk in range(15)].index(d)
            assert abs(st[k] - val[m]) < 1e-14


# -------------------------------------------------------------- ILU(0) ---

def lower_matrix(orc, N, L):
    ic = orc.interior_coords(N)
    cidx = {tuple(int(v) for v in p): i for i, p in enumerate(ic)}
    n = len(ic)
    Lm = np.eye(n)
    for d in range(7):
        dv = np.array([orc.lib().orc_dir(d, c) for c in range(3)])
        for i, p in enumerate(ic):
            j = cidx.get(tuple(int(v) for v in p + dv))
            if j is not None:
                Lm[i, j] = L[d, i]
    return Lm


def interior_block(orc, A, N):
    S = orc.to_scipy(A, N)
    ids, _ = orc.interior_ids(N)
    inter = np.nonzero(ids >= 0)[0]
    return S[inter][:, inter].toarray()


@pytest.mark.parametrize("level", [3, 4, 5])
def test_ilu_defining_identity(orc, level):
    """(L D L^T)_ij = (R_t A R_t^T)_ij on the sparsity pattern (Sec. 3), with L
    unit lower triangular on the pattern: this characterises ILU(0)."""
    N = 2 ** level
    P = si.macro_tet(12)
    A = orc.assemble(P, N, orc.Coeff("sinprod", 1.0, 0.5))
    L, D = orc.ilu0(A, N)
    Att = interior_block(orc, A, N)
    Lm = lower_matrix(orc, N, L)
    pat = Att != 0
    assert np.all((Lm != 0) <= pat | np.eye(len(D), dtype=bool))
    R = Lm @ np.diag(D) @ Lm.T - Att
    assert np.abs(R[pat]).max() < 1e-14 * np.abs(Att).max()
    assert np.all(D > 0)


def test_ilu_level2_single_node(orc):
    """At level 2 the interior is the single point (1,1,1): D = A_c, no L."""
    P = si.macro_tet(13)
    A = orc.assemble(P, 4)
    L, D = orc.ilu0(A, 4)
    st = orc.local_stencil(P, 4, (1, 1, 1))
    assert L.shape == (7, 1) and np.all(L == 0)
    assert abs(D[0] - st[7]) < 1e-15


@pytest.mark.parametrize("level", [2, 3, 4, 5, 6])
def test_algorithm1_equals_ikj(orc, level):
    """The paper's streaming Algorithm 1 reproduces textbook ILU(0)."""
    N = 2 ** level
    P = si.macro_tet(14)
    co = orc.Coeff("kappa_i", ipow=2)
    A = orc.assemble(P, N, co)
    L1, D1 = orc.ilu0(A, N)
    L2, D2 = orc.alg1(P, N, co)
    assert np.abs(L1 - L2).max() < 1e-13
    assert np.abs(D1 - D2).max() < 1e-13 * np.abs(D1).max()


def test_scaling_remark_and_asymptotic_stencil(orc):
    """Remark of Sec. 3: D scales like h, L like 1.  Deep inside the tet the
    factor equals the asymptotic stencil, obtained by Gauss-Seidel iteration of
    the stencil equations from L_c = D_c = 1, L_d = 0 (Sec. 3)."""
    P = si.REFERENCE_TET
    vals = {}
    for level in [5, 6, 7]:
        N = 2 ** level
        A = orc.assemble(P, N)
        L, D = orc.ilu0(A, N)
        ic = orc.interior_coords(N)
        i = int(np.nonzero(np.all(ic == N // 4, axis=1))[0][0])
        vals[level] = (L[:, i].copy(), D[i])
    assert abs(vals[7][1] / vals[6][1] - 0.5) < 1e-10
    assert abs(vals[6][1] / vals[5][1] - 0.5) < 1e-7
    assert np.abs(vals[7][0] - vals[6][0]).max() < 1e-12
    # asymptotic stencil from constant A (stencil at a deep interior point)
    N = 128
    A = orc.local_stencil(P, N, (20, 20, 20))
    W, S, SE, BNW, BN, BC, BE, C = range(8)
    Lv = np.zeros(7); Dc = 1.0
    for _ in range(500):
        bc = A[BC] / Dc
        s = (A[S] - bc * Dc * Lv[BN]) / Dc
        bnw = (A[BNW] - bc * Dc * Lv[SE]) / Dc
        be = (A[BE] - bc * Dc * Lv[W]) / Dc
        w = (A[W] - bc * Dc * Lv[BE] - bnw * Dc * Lv[BN] - s * Dc * Lv[SE]) / Dc
        bn = (A[BN] - bc * Dc * Lv[S] - be * Dc * Lv[SE] - bnw * Dc * Lv[W]) / Dc
        se = (A[SE] - bc * Dc * Lv[BNW] - be * Dc * Lv[BN] - s * Dc * Lv[W]) / Dc
        Lv = np.array([w, s, se, bnw, bn, bc, be])
        Dc = A[C] - Dc * (Lv ** 2).sum()
    assert np.abs(Lv - vals[7][0]).max() < 1e-12
    assert abs(Dc - vals[7][1]) < 1e-12 * Dc


# ------------------------------------------------------------ samples ---

def test_sample_sets(orc):
    """S_d of Sec. 4.1: points congruent to 1 - d modulo the stride, with p+d
    interior; the c direction starts at (1,1,1), w is shifted in x and be in z
    (caption of the sample-set figure)."""
    N, stride = 32, 4
    ic = orc.interior_coords(N)
    for d in range(8):
        dv = np.array([orc.lib().orc_dir(d, c) for c in range(3)])
        S = orc.sample_set(N, d, stride)
        pts = ic[S]
        assert len(S) > 0
        assert np.all((pts - (1 - dv)) % stride == 0)
        q = pts + dv
        assert np.all(q.min(1) >= 1) and np.all(q.sum(1) <= N - 1)
        # completeness: every qualifying interior point is a sample
        ok = np.all((ic - (1 - dv)) % stride == 0, axis=1) & np.all(ic + dv >= 1, axis=1) & \
            ((ic + dv).sum(1) <= N - 1)
        assert set(np.nonzero(ok)[0]) == set(S.tolist())
    assert np.all(ic[orc.sample_set(N, 7, stride)] % stride == 1)
    assert np.all(ic[orc.sample_set(N, 0, stride)][:, 0] % stride == 2)
    assert np.all(ic[orc.sample_set(N, 6, stride)][:, 2] % stride == 2)


# -------------------------------------------------------------- fit -----

def test_fit_reproduces_polynomials(orc):
    """A target inside the tensor space is reproduced: exactly by plain least
    squares, to the ridge bias by the regularised fit."""
    N, deg = 32, [3, 3, 3]
    ic = orc.interior_coords(N).astype(float) / N
    f = 1.0 + 0.3 * ic[:, 0] - 0.2 * ic[:, 1] ** 2 + 0.7 * ic[:, 0] * ic[:, 2] ** 3 - 0.1 * ic[:, 1] ** 3 * ic[:, 0]
    Lfac = np.tile(f, (7, 1))
    Dfac = 1.0 / f
    for ridge, tol in [(0.0, 1e-10), (1e-6, 2e-6)]:
        coefs = orc.fit_surrogates(N, Lfac, Dfac, deg, ridge=ridge)
        Ls, Dinv = orc.eval_surrogates(N, deg, coefs)
        ok = Ls[0] != 0  # V2 mask zeroes points whose west neighbour is boundary
        assert np.abs(Ls[0][ok] - f[ok]).max() < tol
        assert np.abs(Dinv - f).max() < tol


def test_fit_error_decreases_with_degree(orc):
    """Sec. 4.2 (discrete L2 error figure): higher degree, smaller error."""
    pr = orc.Problem(si.macro_tet(1), 5)
    errs = []
    for deg in [0, 2, 4, 6]:
        pr.set_degree(deg)
        mask = pr.L != 0
        eL = np.linalg.norm((pr.Ls - pr.L)[mask]) / np.linalg.norm(pr.L[mask])
        eD = np.linalg.norm(pr.Dinv_s - 1 / pr.D) / np.linalg.norm(1 / pr.D)
        errs.append((eL, eD))
    for a, b in zip(errs, errs[1:]):
        assert b[0] < a[0] and b[1] < a[1]
    assert errs[-1][0] < 0.2 * errs[0][0]


def test_ridge_fit_is_solver_independent(orc):
    """The regularised problem is well posed: an SVD-based and a QR-based solve
    agree on the surrogate values at every interior point."""
    N, deg = 32, [6, 6, 6]
    pr = orc.Problem(si.macro_tet(1), 5)
    ic = orc.interior_coords(N).astype(float)
    Vall = orc.basis_rows(N, deg, ic)
    for d in [0, 5, 7]:
        S = orc.sample_set(N, d, 1)
        t = pr.L[d][S] if d < 7 else 1.0 / pr.D[S]
        V = Vall[S]
        M = V.shape[1]
        lam = 1e-6 * np.sqrt(len(S))
        Va = np.vstack([V, lam * np.eye(M)]); ta = np.concatenate([t, np.zeros(M)])
        c1 = np.linalg.lstsq(Va, ta, rcond=None)[0]
        Q, R = np.linalg.qr(Va)
        c2 = sl.solve_triangular(R, Q.T @ ta)
        f1, f2 = Vall @ c1, Vall @ c2
        assert np.abs(f1 - f2).max() < 1e-10 * np.abs(f1).max()


# ----------------------------------------------------------- smoother ---

def test_smoother_solves_level2(orc):
    """With exact factors at level 2 (one interior point) one sweep solves."""
    P = si.macro_tet(15)
    A = orc.assemble(P, 4)
    L, D = orc.ilu0(A, 4)
    x = si.boundary_data(2, 16)
    b = si.rhs(2, 17)
    orc.smooth(A, 4, L, 1 / D, x, b, 1)
    _, rn = orc.residual(A, 4, x, b)
    assert rn < 1e-14


@pytest.mark.parametrize("level", [3, 4])
def test_smoother_matches_dense_formula(orc, level):
    """One sweep equals x + R_t^T (L D L^T)^{-1} R_t (b - A x), Sec. 2.1 and
    Algorithm 2, computed with dense linear algebra."""
    N = 2 ** level
    P = si.macro_tet(18)
    pr = orc.Problem(P, level, orc.Coeff("sinprod", 1.0, 0.5), deg=3)
    S = orc.to_scipy(pr.A, N)
    ids, _ = orc.interior_ids(N)
    inter = ids >= 0
    x0 = si.boundary_data(level, 19)
    b = si.rhs(level, 20)
    for Lf, Dinv in [pr.exact_factors(), pr.surrogate_factors()]:
        Lm = lower_matrix(orc, N, Lf)
        C = Lm @ np.diag(1.0 / Dinv) @ Lm.T
        r = (b - S @ x0)[inter]
        expect = x0.copy()
        expect[inter] += np.linalg.solve(C, r)
        x = orc.smooth(pr.A, N, Lf, Dinv, x0.copy(), b, 1)
        assert np.abs(x - expect).max() < 1e-12 * np.abs(expect).max()


def test_fixed_point_and_symmetry(orc):
    """The exact solution is a fixed point of a sweep; C^{-1} is symmetric."""
    level, N = 4, 16
    pr = orc.Problem(si.macro_tet(21), level, deg=4)
    Ls, Dinv = pr.surrogate_factors()
    S = orc.to_scipy(pr.A, N)
    ids, _ = orc.interior_ids(N)
    inter = np.nonzero(ids >= 0)[0]
    xs = si.boundary_data(level, 22)
    b = S @ xs
    x = orc.smooth(pr.A, N, Ls, Dinv, xs.copy(), b, 1)
    assert np.abs(x - xs).max() < 1e-12
    u = np.zeros(len(xs)); u[inter] = si.rhs(level, 23)[inter]
    v = np.zeros(len(xs)); v[inter] = si.rhs(level, 24)[inter]
    Cu = orc.smooth(pr.A, N, Ls, Dinv, np.zeros(len(xs)), u, 1)
    Cv = orc.smooth(pr.A, N, Ls, Dinv, np.zeros(len(xs)), v, 1)
    # with x = 0 and zero boundary, one sweep returns C^{-1} b
    assert abs(Cu @ v - u @ Cv) < 1e-12 * abs(Cu @ v)


def test_exact_ilu_contracts(orc):
    """With exact ILU(0) the eigenvalues of C^{-1} A_tt lie in (0, 2), so the
    smoothed Richardson iteration converges (Sec. 2.1)."""
    level, N = 4, 16
    pr = orc.Problem(si.macro_tet(25), level)
    Att = interior_block(orc, pr.A, N)
    Lm = lower_matrix(orc, N, pr.L)
    C = Lm @ np.diag(pr.D) @ Lm.T
    ev = np.linalg.eigvals(np.linalg.solve(C, Att)).real
    assert ev.min() > 0 and ev.max() < 2


def test_outer_solves_reach_tolerance(orc):
    level, N = 4, 16
    pr = orc.Problem(si.macro_tet(26), level, orc.Coeff("sinprod", 1.0, 0.5), deg=4)
    Ls, Dinv = pr.surrogate_factors()
    b = si.rhs(level, 27)
    S = orc.to_scipy(pr.A, N)
    ids, _ = orc.interior_ids(N)
    inter = np.nonzero(ids >= 0)[0]
    xref = np.zeros(len(b))
    xref[inter] = spla.spsolve(S[inter][:, inter].tocsc(), b[inter])
    x1 = np.zeros(len(b))
    it1, rel1 = orc.richardson(pr.A, N, Ls, Dinv, x1, b, 1e-8)
    x2 = np.zeros(len(b))
    it2, rel2 = orc.pcg(pr.A, N, Ls, Dinv, x2, b, 1e-8)
    assert it1 > 0 and rel1 < 1e-8 and it2 > 0 and rel2 < 1e-8
    assert it2 < it1
    for x in (x1, x2):
        assert np.abs(x - xref).max() < 1e-6 * np.abs(xref).max()


# ------------------------------------------- symmetric Gauss-Seidel (Sec. 4.2)

@pytest.mark.parametrize("level,kind", [(3, "const"), (4, "sinprod")])
def test_sgs_factor_form_is_textbook_sgs(orc, level, kind):
    """The L D L^T form of the comparison smoother (L^p_d = a(p,p+d)/a(p+d,p+d),
    D^p = a(p,p)) applied by Algorithm 2 equals a symmetric Gauss-Seidel
    sweep written out point by point."""
    N = 2 ** level
    co = {"const": orc.Coeff(), "sinprod": orc.Coeff("sinprod", 1.0, 0.5)}[kind]
    pr = orc.Problem(si.macro_tet(60), level, co, factor="sgs")
    x0 = si.boundary_data(level, 61)
    b = si.rhs(level, 62)
    xa = orc.smooth(pr.A, N, pr.L, 1.0 / pr.D, x0.copy(), b, 2)
    xb = x0.copy()
    for _ in range(2):
        orc.sgs_sweep(pr.A, N, xb, b)
    assert np.abs(xa - xb).max() < 1e-12 * np.abs(xb).max()


def test_sgs_factors_reproduce_the_splitting(orc):
    """L D L^T of the SGS factors is (D + E) D^{-1} (D + E^T), with D and E the
    diagonal and strictly lower part of the interior block (dense algebra)."""
    level, N = 3, 8
    pr = orc.Problem(si.macro_tet(63), level, orc.Coeff("kappa_i", 0.0, 0.0, 2), factor="sgs")
    Att = interior_block(orc, pr.A, N)
    Dm = np.diag(np.diag(Att))
    E = np.tril(Att, -1)
    want = (Dm + E) @ np.linalg.inv(Dm) @ (Dm + E).T
    Lm = lower_matrix(orc, N, pr.L)
    got = Lm @ np.diag(pr.D) @ Lm.T
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_exact_ilu_beats_sgs(orc):
    """With exact factors the ILU(0) smoother contracts faster than symmetric
    Gauss-Seidel on the same problem (the comparison of Sec. 4.2)."""
    level, N = 4, 16
    P = si.macro_tet(64)
    ilu = orc.Problem(P, level)
    sgs = orc.Problem(P, level, factor="sgs")
    Att = interior_block(orc, ilu.A, N)
    rho = []
    for pr in (ilu, sgs):
        Lm = lower_matrix(orc, N, pr.L)
        C = Lm @ np.diag(pr.D) @ Lm.T
        ev = np.linalg.eigvals(np.eye(len(Att)) - np.linalg.solve(C, Att))
        rho.append(np.abs(ev).max())
    assert rho[0] < rho[1] < 1


# ----------------------------------------------------- boundary variant ---

@pytest.mark.parametrize("level", [2, 3, 4])
def test_cell_boundary_mask_is_the_points_with_an_outside_neighbour(orc, level):
    """V1 (Sec. 4.1): the cell-boundary points are the interior points with a
    neighbour in D outside the interior; checked by brute force."""
    N = 2 ** level
    dirs = [(-1, 0, 0), (0, -1, 0), (1, -1, 0), (-1, 1, -1), (0, 1, -1), (0, 0, -1), (1, 0, -1),
            (1, 0, 0), (0, 1, 0), (-1, 1, 0), (1, -1, 1), (0, -1, 1), (0, 0, 1), (-1, 0, 1)]
    inside = lambda x, y, z: x >= 1 and y >= 1 and z >= 1 and x + y + z <= N - 1
    want = np.array([any(not inside(x + a, y + b, z + c) for a, b, c in dirs)
                     for x, y, z in orc.interior_coords(N)])
    assert np.array_equal(orc.cell_boundary_mask(N), want)
    # O(N^2): every interior point at level 2 and 3, a thin shell above
    if level == 4:
        assert want.sum() < 0.75 * len(want)


def test_v1_with_exact_factors_is_the_exact_smoother(orc):
    """With the surrogate replaced by the exact factors, V1 changes nothing;
    with zero surrogates, exactly the cell-boundary points carry the stored
    factors L^p_d and 1/D^p (Sec. 4.1, Alg. 1)."""
    pr = orc.Problem(si.macro_tet(31), 4)
    L1, D1 = orc.v1_factors(pr.N, pr.L, 1.0 / pr.D, pr.L, pr.D)
    assert np.array_equal(L1, pr.L) and np.array_equal(D1, 1.0 / pr.D)
    Lx, Dx = orc.v1_factors(pr.N, np.zeros_like(pr.L), np.zeros_like(pr.D), pr.L, pr.D)
    m = orc.cell_boundary_mask(pr.N)
    assert np.array_equal(Lx[:, m], pr.L[:, m]) and not Lx[:, ~m].any()
    assert np.array_equal(Dx[m], 1.0 / pr.D[m]) and not Dx[~m].any()


def test_v1_at_level_2_solves_in_one_sweep_whatever_the_surrogate(orc):
    """Level 2 has one interior point, on the cell boundary, whose exact
    factor is D = A_c.  V1 stores 1/D there, so one V1 sweep solves the
    problem exactly however wrong the surrogate is.  The same sweep with the
    surrogate's D~^-1 (the planted mistake of not using the stored centre)
    does not."""
    P = si.macro_tet(32)
    pr = orc.Problem(P, 2)
    N = pr.N
    bad_L = np.full_like(pr.L, 0.3)
    bad_Dinv = 0.5 / pr.D
    x0 = si.boundary_data(2, 33)
    b = si.rhs(2, 34)
    L1, D1 = orc.v1_factors(N, bad_L, bad_Dinv, pr.L, pr.D)
    x = orc.smooth(pr.A, N, L1, D1, x0.copy(), b, 1)
    assert orc.residual(pr.A, N, x, b)[1] <= 1e-14 * max(1.0, np.abs(b).max())
    wrong = orc.smooth(pr.A, N, L1, bad_Dinv, x0.copy(), b, 1)
    assert orc.residual(pr.A, N, wrong, b)[1] > 1e-3 * orc.residual(pr.A, N, x0, b)[1]

def test_local_ldlt_apply_recovers_the_residual_of_one_sweep(orc):
    """One oracle sweep x1 = x0 + C~^-1 r; the point-local (L~ D~ L~^T w)_p of
    w = x1 - x0, evaluated from the surrogate polynomials, equals the point's
    residual r_p at every interior point, and local_residual equals the
    assembled residual.  A dropped backward term is caught."""
    level, deg = 4, [3, 3, 3]
    P = si.macro_tet(35)
    co = orc.Coeff("sinprod", 1.0, 0.5)
    pr = orc.Problem(P, level, co, deg=deg)
    N = pr.N
    x0 = si.boundary_data(level, 36)
    b = si.rhs(level, 37)
    Ls, Dinv = pr.surrogate_factors()
    x1 = orc.smooth(pr.A, N, Ls, Dinv, x0.copy(), b, 1)
    r, _ = orc.residual(pr.A, N, x0, b)
    w = x1 - x0
    at = lambda v: (lambda q: v[orc.index(N, *q)])
    cache = {}
    worst = 0.0
    for q in map(tuple, orc.interior_coords(N)):
        got = orc.ldlt_apply_at(N, deg, pr.coefs, at(w), q, cache)
        worst = max(worst, abs(got - r[orc.index(N, *q)]))
        assert abs(orc.local_residual(P, N, co, at(x0), at(b), q) - r[orc.index(N, *q)]) < 1e-12
    assert worst < 1e-11 * np.abs(r).max()
    # planted mistake: w with one backward term dropped (w at its neighbour perturbed)
    q0 = (2, 2, 2)
    wp = w.copy()
    wp[orc.index(N, 3, 2, 2)] *= 1.01
    assert abs(orc.ldlt_apply_at(N, deg, pr.coefs, at(wp), q0) - r[orc.index(N, *q0)]) > 1e-6 * np.abs(r).max()
