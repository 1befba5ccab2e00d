"""GPU outer solves (smoothed Richardson with defect correction, and PCG)
against the CPU oracle: same surrogate, same stopping rule, the solution of
the assembled system."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import seeded_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_15280_gb300 as g
    g.build()
    return g


def exact_solution(orc, pr, N, b, xbd):
    S = orc.to_scipy(pr.A, N)
    ids, _ = orc.interior_ids(N)
    inter = np.nonzero(ids >= 0)[0]
    bnd = np.nonzero(ids < 0)[0]
    x = xbd.copy()
    rhs = b[inter] - S[inter][:, bnd] @ xbd[bnd]
    x[inter] = spla.spsolve(S[inter][:, inter].tocsc(), rhs)
    return x


@pytest.mark.parametrize("prec,kernel", [("F64", "AUTO"), ("MIXED", "SLAB"), ("MIXED", "BAND"), ("MIXED", "PACKED")])
@pytest.mark.parametrize("method", ["RICHARDSON", "PCG"])
def test_solve_reaches_tolerance(g, orc, prec, method, kernel):
    level, deg, N = 4, 4, 16
    P = si.macro_tet(101)
    co = ("sinprod", 1.0, 0.5, 0)
    pr = orc.Problem(P, level, orc.Coeff(*co), deg=deg)
    t = g.Tet(P, level, coeff=g.make_coeff(*co), poly_degree=deg, precision=getattr(g, prec),
              kernel=getattr(g, "KERNEL_" + kernel))
    t.import_surrogate(pr.coefs)
    b = si.rhs(level, 102)
    xbd = np.zeros(len(b))
    ids, _ = orc.interior_ids(N)
    xbd[ids < 0] = si.boundary_data(level, 103)[ids < 0]  # Dirichlet data on the boundary
    x = torch.tensor(xbd, dtype=torch.float64, device="cuda")
    it, rel, ok = t.solve(x, torch.tensor(b, dtype=torch.float64, device="cuda"), getattr(g, method), 1e-8, 5000)
    assert ok and rel < 1e-8
    xs = exact_solution(orc, pr, N, b, xbd)
    xg = x.cpu().numpy()
    assert np.abs(xg - xs).max() < 1e-6 * np.abs(xs).max()
    assert np.array_equal(xg[ids < 0], xbd[ids < 0])  # boundary untouched
    # the oracle's own iteration, same surrogate and stopping rule
    Ls, Dinv = pr.surrogate_factors()
    xo = xbd.copy()
    ito, relo = (orc.richardson if method == "RICHARDSON" else orc.pcg)(pr.A, N, Ls, Dinv, xo, b, 1e-8)
    assert abs(it - ito) <= (0 if prec == "F64" else 2)


def test_pcg_beats_richardson_and_fp64_matches_mixed(g, orc):
    level, deg = 5, 4
    P = si.macro_tet(104)
    t64 = g.Tet(P, level, coeff=g.make_coeff("const"), poly_degree=deg, precision=g.F64)
    tmx = g.Tet(P, level, coeff=g.make_coeff("const"), poly_degree=deg, precision=g.MIXED)
    b = torch.tensor(si.rhs(level, 105), dtype=torch.float64, device="cuda")
    res = {}
    for name, t in [("f64", t64), ("mixed", tmx)]:
        for m in ["RICHARDSON", "PCG"]:
            x = torch.zeros_like(b)
            it, rel, ok = t.solve(x, b, getattr(g, m), 1e-8, 20000)
            assert ok and rel < 1e-8
            res[(name, m)] = (it, x.cpu().numpy())
    assert res[("f64", "PCG")][0] < res[("f64", "RICHARDSON")][0]
    # FP32 sweeps with FP64 defect correction reach the same solution
    a, c = res[("f64", "RICHARDSON")][1], res[("mixed", "RICHARDSON")][1]
    assert np.abs(a - c).max() < 1e-6 * np.abs(a).max()
    assert abs(res[("f64", "RICHARDSON")][0] - res[("mixed", "RICHARDSON")][0]) <= 3


def test_solve_reports_nonconvergence(g):
    t = g.Tet(si.macro_tet(106), 5, poly_degree=3, precision=g.MIXED)
    b = torch.tensor(si.rhs(5, 107), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    it, rel, ok = t.solve(x, b, g.RICHARDSON, 1e-12, 3)
    assert not ok and it == 3 and rel > 1e-12


@pytest.mark.parametrize("method", ["RICHARDSON", "PCG"])
def test_ilu_smoother_beats_sgs(g, orc, method):
    """The comparison of Sec. 4.2 on one macro-tet: the surrogate ILU(0)
    smoother needs fewer iterations than surrogate symmetric Gauss-Seidel,
    and both reach the same solution."""
    level = 5
    P = si.macro_tet(108)
    co = g.make_coeff("sinprod", 1.0, 0.5)
    b = torch.tensor(si.rhs(level, 109), dtype=torch.float64, device="cuda")
    res = {}
    for name, factor in [("ilu", g.FACTOR_ILU0), ("sgs", g.FACTOR_SGS)]:
        t = g.Tet(P, level, coeff=co, poly_degree=4, precision=g.MIXED, factor=factor)
        x = torch.zeros_like(b)
        it, rel, ok = t.solve(x, b, getattr(g, method), 1e-8, 20000)
        assert ok and rel < 1e-8
        res[name] = (it, x.cpu().numpy())
    assert res["ilu"][0] < res["sgs"][0]
    a, c = res["ilu"][1], res["sgs"][1]
    assert np.abs(a - c).max() < 1e-6 * np.abs(a).max()
