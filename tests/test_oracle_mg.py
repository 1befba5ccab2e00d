"""Pins of the oracle's multigrid (oracle/mg.py) against the mathematics of
nested P1 spaces and against the convergence factors printed in Table 2 of
arXiv 2210.15280 (appendix).

Table 2 pins the whole chain at once: micro-mesh, assembly, exact ILU(0),
the Algorithm 2 smoother, symmetric Gauss-Seidel and the grid transfer.  A
dropped term or a wrong sign in any of them moves rho far outside the printed
two digits.
"""
import os

import numpy as np
import pytest

import seeded_inputs as si

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_table2():
    shapes = {}
    for ln in open(os.path.join(GOLDEN, "table2_shapes.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        name, *v = ln.split()
        shapes.setdefault(name, []).append([float(t) for t in v])
    rows = []
    for ln in open(os.path.join(GOLDEN, "table2_mg_rates.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        name, pi, rg, ri, ng, ni = ln.split()
        rows.append((name, [int(c) for c in pi], rg, ri, int(ng), int(ni)))
    return {k: np.array(v) for k, v in shapes.items()}, rows


def permuted(P, pi):
    """Vertex i goes to position pi(i) (the reading of the table's notation)."""
    Q = np.zeros_like(P)
    for i in range(4):
        Q[pi[i] - 1] = P[i]
    return Q


def printed_tol(s, rel):
    """Half a unit of the last printed digit plus a relative margin for the
    finite power iteration."""
    dec = len(s.split(".")[1]) if "." in s else 0
    return 0.5 * 10.0 ** (-dec) + rel * float(s)


@pytest.fixture(scope="module")
def mg(orc):
    from oracle import mg as M
    return M


@pytest.mark.parametrize("Nc", [2, 4, 8])
def test_prolongation_interpolates_affine_functions(orc, mg, Nc):
    """Nested P1 spaces: an affine function is its own interpolant, and the
    hat functions form a partition of unity."""
    Pm = mg.prolongation(Nc)
    cc, cf = orc.coords(Nc).astype(float), orc.coords(2 * Nc).astype(float)
    a = np.array([0.3, -1.7, 2.2])
    u_c = cc @ a + 0.9
    u_f = (cf / 2.0) @ a + 0.9
    assert np.abs(Pm @ u_c - u_f).max() < 1e-13
    assert np.abs(np.asarray(Pm.sum(axis=1)).ravel() - 1.0).max() < 1e-14
    # nodes shared by both grids take the coarse value unchanged
    for k in [0, len(cc) // 3, len(cc) - 1]:
        x, y, z = orc.coords(Nc)[k]
        row = Pm.getrow(orc.index(2 * Nc, 2 * x, 2 * y, 2 * z)).toarray().ravel()
        e = np.zeros(len(cc)); e[k] = 1.0
        assert np.array_equal(row, e)


@pytest.mark.parametrize("level", [3, 4])
def test_galerkin_identity(orc, mg, level):
    """For constant kappa on an affine tet the coarse stiffness matrix is the
    Galerkin product P^T A_f P of the fine one (nested P1 spaces)."""
    P = si.macro_tet(11)
    Nc = 2 ** (level - 1)
    Af = orc.to_scipy(orc.assemble(P, 2 * Nc, orc.Coeff("const", 2.5)), 2 * Nc)
    Ac = orc.to_scipy(orc.assemble(P, Nc, orc.Coeff("const", 2.5)), Nc)
    Pm = mg.prolongation(Nc)
    G = (Pm.T @ Af @ Pm).toarray()
    assert np.abs(G - Ac.toarray()).max() < 1e-12 * np.abs(Ac).max()


def test_vcycle_on_the_coarsest_level_solves(orc, mg):
    H = mg.Hierarchy(si.macro_tet(12), 3, coarsest=3)
    lv = H.lv[3]
    b = si.rhs(3, 13)
    x = si.boundary_data(3, 14)
    H.vcycle(3, x, b)
    r, rn = orc.residual(lv.A, lv.N, x, b)
    assert rn < 1e-12 * np.linalg.norm(b[lv.inner])


def test_vcycle_reduces_error_and_is_linear(orc, mg):
    """A V-cycle is an affine map with fixed point the solution: from x* it
    stays there, and its error propagation contracts."""
    H = mg.Hierarchy(si.macro_tet(15), 4)
    lv = H.lv[4]
    rng = np.random.default_rng(16)
    xs = np.zeros(orc.num_nodes(lv.N)); xs[lv.inner] = rng.uniform(-1, 1, lv.nint)
    A = orc.to_scipy(lv.A, lv.N)
    b = A @ xs
    x = xs.copy()
    H.vcycle(4, x, b)
    assert np.abs(x - xs).max() < 1e-12
    x = np.zeros_like(xs)
    e0 = np.linalg.norm(xs)
    H.vcycle(4, x, b)
    assert np.linalg.norm(x - xs) < 0.2 * e0


@pytest.fixture(scope="module")
def table2():
    return load_table2()


def _rho(orc, mg, table2, row, smoother):
    shapes, _ = table2
    name, pi = row[0], row[1]
    _, nint = orc.interior_ids(64)
    e0 = np.random.default_rng(5).uniform(-1, 1, nint)
    H = mg.Hierarchy(permuted(shapes[name], pi), 6, smoother=smoother)
    rho, _ = H.rate(e0)
    return rho


ROWS = load_table2()[1]


@pytest.mark.parametrize("row", ROWS, ids=[f"{r[0]}-{''.join(map(str, r[1]))}" for r in ROWS])
def test_table2_ilu_rates(orc, mg, table2, row):
    """rho of the ILU(0)-smoothed V(3,3)-cycle, levels 2..6, 20 power steps."""
    rho = _rho(orc, mg, table2, row, "ilu")
    assert abs(rho - float(row[3])) <= printed_tol(row[3], 0.03), (rho, row)


GS_ROWS = [r for r in ROWS if not (r[0] == "spade" and r[1] == [2, 3, 4, 1])]


@pytest.mark.parametrize("row", GS_ROWS, ids=[f"{r[0]}-{''.join(map(str, r[1]))}" for r in GS_ROWS])
def test_table2_gs_rates(orc, mg, table2, row):
    """rho with symmetric Gauss-Seidel smoothing.  The 20-step power
    iteration leaves more spread here (clustered error modes), hence the
    wider margin.  The Spade (2 3 4 1) entry is left out: its printed 0.055
    fits none of the 24 orders (they give 0.075 to 0.20)."""
    rho = _rho(orc, mg, table2, row, "sgs")
    assert abs(rho - float(row[2])) <= printed_tol(row[2], 0.15), (rho, row)


def test_table2_counts_follow_from_rates(table2):
    """The table's iteration counts are ceil(log(1e-6) / log(rho)) of its own
    rates, so they carry no information beyond rho."""
    for _, _, rg, ri, ng, ni in table2[1]:
        for r, n in [(float(rg), ng), (float(ri), ni)]:
            assert n == int(np.ceil(np.log(1e-6) / np.log(r)))


def test_table2_pin_catches_planted_mistakes(orc, mg, table2):
    """The Table 2 pin is sharp: plausible mistakes planted in the oracle's
    chain move the Regular tet's rate outside the tolerance the pin allows
    around the printed 0.025."""
    shapes, _ = table2
    P = shapes["regular"]
    _, nint = orc.interior_ids(64)
    e0 = np.random.default_rng(5).uniform(-1, 1, nint)
    tol = printed_tol("0.025", 0.03)
    exact, _ = mg.Hierarchy(P, 6).rate(e0)
    assert abs(exact - 0.025) <= tol

    def rate(make):
        fac = {}
        for l in range(3, 7):
            A = orc.assemble(P, 2 ** l)
            fac[l] = make(A, 2 ** l)
        return mg.Hierarchy(P, 6, factors=fac).rate(e0)[0]

    def ilu(A, N):
        L, D = orc.ilu0(A, N)
        return L, 1.0 / D

    planted = {
        # the ILU recursion without its correction sums (= symmetric Gauss-Seidel)
        "dropped correction terms": lambda A, N: (orc.sgs_factors(A, N)[0], 1.0 / orc.sgs_factors(A, N)[1]),
        # two directions of the factor exchanged (w and s)
        "transposed directions": lambda A, N: (ilu(A, N)[0][[1, 0, 2, 3, 4, 5, 6]].copy(), ilu(A, N)[1]),
        # the bc entry of the factor dropped
        "dropped bc term": lambda A, N: (ilu(A, N)[0] * np.array([1, 1, 1, 1, 1, 0, 1.0])[:, None], ilu(A, N)[1]),
        # the diagonal off by 10 %
        "scaled diagonal": lambda A, N: (ilu(A, N)[0], ilu(A, N)[1] / 1.1),
    }
    for name, make in planted.items():
        rho = rate(make)
        assert abs(rho - 0.025) > tol, (name, rho)


def test_height_sweep_follows_the_paper(orc, mg):
    """The paper's height study (Sec. 4.2, the figure on a trirectangular tet
    whose top vertex sinks): with symmetric Gauss-Seidel smoothing the
    V(3,3)-cycle rate degenerates as the height shrinks; with ILU(0) it stays
    robust and tends to an exact solver; the ratio log(rho_ILU)/log(rho_SGS),
    the extra cycles SGS needs, grows without bound."""
    _, nint = orc.interior_ids(64)
    e0 = np.random.default_rng(5).uniform(-1, 1, nint)
    ilu, sgs = [], []
    for h in [1.0, 0.25, 1.0 / 16]:
        P = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, h]], dtype=float)
        ilu.append(mg.Hierarchy(P, 6, smoother="ilu").rate(e0)[0])
        sgs.append(mg.Hierarchy(P, 6, smoother="sgs").rate(e0)[0])
    assert sgs[0] < sgs[1] < sgs[2] and sgs[2] > 0.7, sgs
    assert ilu[0] > ilu[1] > ilu[2] and ilu[0] < 0.05 and ilu[2] < 1e-3, ilu
    ratio = [np.log(a) / np.log(b) for a, b in zip(ilu, sgs)]
    assert ratio[0] < ratio[1] < ratio[2] and ratio[2] > 20, ratio
