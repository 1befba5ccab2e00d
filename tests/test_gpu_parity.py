"""GPU parity of the sweep kernels against the CPU oracle (element by element).

Each case draws its macro-tetrahedron, right-hand side and start vector from
seeded_inputs, fits the surrogate with the oracle, imports the oracle's
coefficients into the library (so both sides evaluate the same polynomials)
and compares the smoothed vectors:
  * F64: within 1e-12 relative (max abs difference / max abs value),
  * F32 and MIXED: within 1e-5 relative per sweep from the same start vector.
"""
import numpy as np
import pytest

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


_cache = {}


def problem(orc, level, seed, kind, deg):
    key = (level, seed, kind, tuple(np.atleast_1d(deg)))
    if key not in _cache:
        co = {"const": ("const", 1.0, 0.0, 0), "sinprod": ("sinprod", 1.0, 0.5, 0),
              "kappa_i": ("kappa_i", 0.0, 0.0, 2)}[kind]
        P = si.macro_tet(seed)
        _cache[key] = (P, co, orc.Problem(P, level, orc.Coeff(*co), deg=deg))
    return _cache[key]


def gpu_tet(g, P, level, co, deg, prec, coefs, slabs=0):
    t = g.Tet(P, level, coeff=g.make_coeff(*co), poly_degree=deg if np.isscalar(deg) else 0,
              deg=deg, precision=prec, slabs=slabs)
    t.import_surrogate(coefs)
    return t


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def dev(v, dtype):
    return torch.tensor(np.ascontiguousarray(v), dtype=dtype, device="cuda")


@pytest.mark.parametrize("level,kind,deg", [(2, "const", 2), (3, "const", 3), (4, "sinprod", 4), (5, "const", 4),
                                            (5, "sinprod", 6), (6, "kappa_i", 5), (6, "sinprod", [2, 3, 4])])
def test_f64_sweeps_match_oracle(g, orc, level, kind, deg):
    P, co, pr = problem(orc, level, 41 + level, kind, deg)
    N = 2 ** level
    t = gpu_tet(g, P, level, co, deg, g.F64, pr.coefs)
    x0 = si.boundary_data(level, 42)
    b = si.rhs(level, 43)
    xo = x0.copy()
    Ls, Dinv = pr.surrogate_factors()
    _, no = orc.smooth(pr.A, N, Ls, Dinv, xo, b, 3, want_norms=True)
    xd = dev(x0, torch.float64)
    bd = dev(b, torch.float64)
    ng = t.smooth(xd, bd, 3, norms=True)
    xg = xd.cpu().numpy()
    assert rel(xg, xo) < 1e-12
    assert np.allclose(ng, no, rtol=1e-12)


@pytest.mark.parametrize("prec", ["F32", "MIXED"])
@pytest.mark.parametrize("level,kind,deg", [(4, "const", 4), (5, "sinprod", 6), (6, "const", 6), (7, "sinprod", 6)])
def test_reduced_precision_per_sweep(g, orc, prec, level, kind, deg):
    """Each sweep, started from the oracle's current iterate, lands within
    1e-5 (relative) of the oracle's next iterate."""
    P, co, pr = problem(orc, level, 51 + level, kind, deg)
    N = 2 ** level
    p = getattr(g, prec)
    t = gpu_tet(g, P, level, co, deg, p, pr.coefs)
    dt = torch.float32 if p == g.F32 else torch.float64
    x = si.boundary_data(level, 52)
    b = si.rhs(level, 53)
    Ls, Dinv = pr.surrogate_factors()
    bd = dev(b, dt)
    for k in range(3):
        xn = orc.smooth(pr.A, N, Ls, Dinv, x.copy(), b, 1)
        xd = dev(x, dt)
        t.smooth(xd, bd, 1)
        assert rel(xd.cpu().numpy().astype(np.float64), xn) < 1e-5
        x = xn


def test_slab_partition_is_bitwise_invariant(g, orc):
    """The result does not depend on how the tet is split into z-slabs."""
    level, deg = 6, 4
    P, co, pr = problem(orc, level, 61, "sinprod", deg)
    x0 = si.boundary_data(level, 62)
    b = si.rhs(level, 63)
    outs = []
    for slabs in [1, 2, 3, 7, 61]:
        t = gpu_tet(g, P, level, co, deg, g.F64, pr.coefs, slabs=slabs)
        xd = dev(x0, torch.float64)
        t.smooth(xd, dev(b, torch.float64), 2)
        outs.append(xd.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("prec", ["F64", "MIXED", "F32"])
def test_residual_matches_oracle(g, orc, prec):
    level = 5
    P, co, pr = problem(orc, level, 71, "sinprod", 3)
    N = 2 ** level
    p = getattr(g, prec)
    t = gpu_tet(g, P, level, co, 3, p, pr.coefs)
    dt = torch.float32 if p == g.F32 else torch.float64
    x = si.boundary_data(level, 72)
    b = si.rhs(level, 73)
    xd, bd = dev(x, dt), dev(b, dt)
    r = torch.zeros_like(xd)
    nrm = t.residual(xd, bd, r)
    ro, no = orc.residual(pr.A, N, x.astype(dt == torch.float32 and np.float32 or np.float64).astype(np.float64),
                          b.astype(dt == torch.float32 and np.float32 or np.float64).astype(np.float64))
    tol = 1e-5 if p == g.F32 else 1e-13
    assert rel(r.cpu().numpy().astype(np.float64), ro) < tol
    assert abs(nrm - no) < tol * no


def test_host_entry_point_matches_device(g, orc):
    level = 5
    P, co, pr = problem(orc, level, 81, "const", 4)
    t = gpu_tet(g, P, level, co, 4, g.MIXED, pr.coefs)
    x0 = si.boundary_data(level, 82)
    b = si.rhs(level, 83)
    xh = x0.copy()
    t.smooth_host(xh, b, 4)
    xd = dev(x0, torch.float64)
    t.smooth(xd, dev(b, torch.float64), 4)
    assert np.array_equal(xh, xd.cpu().numpy())


def test_library_fit_end_to_end(g, orc):
    """Without importing the oracle's coefficients: the library's own set-up
    and sweep agree with the oracle's own fit and sweep to the FP32 bar."""
    level, deg = 6, 6
    P, co, pr = problem(orc, level, 91, "sinprod", deg)
    N = 2 ** level
    t = g.Tet(P, level, coeff=g.make_coeff(*co), poly_degree=deg, precision=g.MIXED)
    x0 = si.boundary_data(level, 92)
    b = si.rhs(level, 93)
    Ls, Dinv = pr.surrogate_factors()
    xo = orc.smooth(pr.A, N, Ls, Dinv, x0.copy(), b, 1)
    xd = dev(x0, torch.float64)
    t.smooth(xd, dev(b, torch.float64), 1)
    assert rel(xd.cpu().numpy(), xo) < 1e-5
