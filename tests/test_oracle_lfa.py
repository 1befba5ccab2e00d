"""Pins of the oracle's local Fourier analysis (oracle/lfa.py) and of the
library's vertex-order choice (ilu_lfa_order, host code, no GPU).

The asymptotic stencil is pinned to the exact ILU(0) deep inside a fine
grid; the smoothing factors to the symmetry of the regular tetrahedron; the
choice of order to the bold entries of the paper's Table 2 through the
oracle's multigrid (itself pinned to that table).
"""
import os

import numpy as np
import pytest

import seeded_inputs as si

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
REGULAR = np.array([[0, 0, 0], [1, 0, 0], [0.5, np.sqrt(3) / 2, 0], [0.5, np.sqrt(3) / 6, np.sqrt(2 / 3)]])


@pytest.fixture(scope="module")
def lfa(orc):
    from oracle import lfa as M
    return M


def shapes():
    out = {}
    for ln in open(os.path.join(GOLDEN, "table2_shapes.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        name, *v = ln.split()
        out.setdefault(name, []).append([float(t) for t in v])
    return {k: np.array(v) for k, v in out.items()}


def bold():
    rows = []
    for ln in open(os.path.join(GOLDEN, "table2_lfa_choice.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        name, pi, rho = ln.split()
        rows.append((name, [int(c) for c in pi], rho))
    return rows


@pytest.mark.parametrize("seed", [None, 21])
def test_asymptotic_stencil_is_the_deep_interior_ilu(orc, lfa, seed):
    """The fixed point of the stencil equations is what the exact ILU(0)
    converges to far from the boundary (checked at level 7)."""
    P = si.REFERENCE_TET if seed is None else si.macro_tet(seed)
    N = 128
    A = orc.assemble(P, N)
    L, D = orc.ilu0(A, N)
    ic = orc.interior_coords(N)
    i = int(np.nonzero(np.all(ic == N // 4, axis=1))[0][0])
    La, Da = lfa.asymptotic_stencil(orc.local_stencil(P, N, (N // 4,) * 3))
    assert np.abs(La - L[:, i]).max() < 1e-10
    assert abs(Da - D[i]) < 1e-10 * D[i]


def test_asymptotic_stencil_scaling(orc, lfa):
    """Remark of Sec. 3: L does not depend on the scale of A, D scales with it."""
    A = lfa.constant_stencil(si.macro_tet(22))
    L1, D1 = lfa.asymptotic_stencil(A)
    L2, D2 = lfa.asymptotic_stencil(8.0 * A)
    assert np.abs(L1 - L2).max() < 1e-13 and abs(D2 / D1 - 8.0) < 1e-12


def test_regular_tet_orders_are_equivalent(lfa):
    """Every vertex order of the regular tetrahedron is a symmetry of it."""
    _, mu, mus = lfa.best_order(REGULAR)
    assert 0.0 < mu < 1.0
    assert np.ptp(mus) < 1e-12


def test_theta_grid(lfa):
    T = lfa.theta_grid(16)
    assert len(T) == 16 ** 3 - 7 ** 3
    assert np.all(np.any(np.abs(T) >= np.pi / 2, axis=1))


@pytest.mark.parametrize("row", bold(), ids=[r[0] for r in bold()])
def test_chosen_order_gives_the_bold_rate(orc, lfa, row):
    """The order picked by the smoothing factor yields, in the oracle's
    V(3,3)-cycle on levels 2..6, the rate the paper prints in bold (for the
    Spindle that is not the best rate of the table: the heuristic picks
    (1 3 2 4) with 0.39 over (1 4 2 3) with 0.35)."""
    from oracle import mg
    name, pi, rho_s = row
    P = shapes()[name]
    perm, mu, _ = lfa.best_order(P)
    _, nint = orc.interior_ids(64)
    e0 = np.random.default_rng(5).uniform(-1, 1, nint)
    rho, _ = mg.Hierarchy(P[perm], 6).rate(e0)
    dec = len(rho_s.split(".")[1])
    assert abs(rho - float(rho_s)) <= 0.5 * 10.0 ** (-dec) + 0.06 * float(rho_s), (perm, rho)


@pytest.fixture(scope="module")
def g():
    import paper_2210_15280_gb300 as G
    G.build()
    return G


@pytest.mark.parametrize("name", ["spindle", "cap", "spade", "regular", "perturbed", "flat"])
def test_library_order_matches_oracle(g, lfa, name):
    P = {"perturbed": si.macro_tet(3, 0.3), "flat": np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 0.05]]),
         "regular": REGULAR}.get(name)
    if P is None:
        P = shapes()[name]
    perm, mu, mus = g.lfa_order(P)
    op, omu, omus = lfa.best_order(P)
    omus = np.array(omus)
    assert np.abs(mus - omus).max() < 1e-10 * omus.max()
    assert abs(mu - omus.min()) < 1e-10 * omus.min()
    assert abs(omus[[list(p) for p in __import__("itertools").permutations(range(4))].index(perm)] - omus.min()) \
        < 1e-10 * omus.min()


def test_setup_uses_the_lfa_order(g):
    """ILU_ORIENT_LFA sets the handle up on the reordered vertices: same
    stencils as a handle given that order explicitly."""
    P = shapes()["spindle"]
    perm, _, _ = g.lfa_order(P)
    a = g.Tet(P, 4, device=-1, orient=g.ORIENT_LFA)
    b = g.Tet(P[perm], 4, device=-1)
    assert a.vertex_order() == perm and b.vertex_order() == [0, 1, 2, 3]
    for p in [(1, 1, 1), (3, 5, 2), (2, 2, 7)]:
        assert np.array_equal(a.stencil(*p), b.stencil(*p))
        assert np.array_equal(a.eval_surrogate(*p), b.eval_surrogate(*p))
    with pytest.raises(g.IluError):
        g.lfa_order(np.zeros((4, 3)))
