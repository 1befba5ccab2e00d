"""Host-side (no GPU) checks of the library: the C ABI loads and exports
every declared symbol, and its FP64 set-up (stencils, streaming ILU(0),
surrogate fit, per-row tables) agrees with the independent CPU oracle."""
import math
import os
import re

import numpy as np
import pytest

import seeded_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    import paper_2210_15280_gb300 as g
    g.build()
    return g


def host_tet(g, P, level, coeff=None, deg=4, **kw):
    return g.Tet(P, level, coeff=coeff, poly_degree=deg, device=-1, **kw)


def test_exports_every_declared_symbol(g):
    hdr = open(os.path.join(ROOT, "include", "ilu.h")).read()
    declared = set(re.findall(r"\b(ilu_[a-z0-9_]+)\s*\(", hdr))
    assert declared, "no declarations parsed"
    L = g.lib()
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared == set(g.EXPORTS)


def test_grid_helpers(g, orc):
    for level in [2, 3, 5, 7]:
        N = 2 ** level
        assert g.num_nodes(level) == math.comb(N + 3, 3) == orc.num_nodes(N)
        assert g.num_interior(level) == math.comb(N - 1, 3)
    for p in [(0, 0, 0), (1, 2, 3), (5, 0, 3), (0, 0, 8)]:
        assert g.index(3, *p) == orc.index(8, *p)
    assert g.index(3, 5, 5, 5) == -1
    assert g.num_nodes(11) == 0


@pytest.mark.parametrize("kind", ["const", "sinprod", "kappa_i"])
def test_stencils_match_oracle(g, orc, kind):
    level, N = 4, 16
    P = si.macro_tet(31)
    co = {"const": ("const", 2.5, 0.0, 0), "sinprod": ("sinprod", 1.0, 0.5, 0), "kappa_i": ("kappa_i", 0.0, 0.0, 3)}[kind]
    t = host_tet(g, P, level, coeff=g.make_coeff(*co), deg=2)
    oc = orc.Coeff(*co)
    for p in orc.interior_coords(N)[::7]:
        a = t.stencil(*p)
        b = orc.local_stencil(P, N, p, oc)
        assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("level,kind", [(3, "const"), (4, "sinprod"), (5, "const"), (5, "sinprod")])
def test_streaming_factorisation_matches_ikj(g, orc, level, kind):
    N = 2 ** level
    P = si.macro_tet(32)
    co = ("sinprod", 1.0, 0.5, 0) if kind == "sinprod" else ("const", 1.0, 0.0, 0)
    t = host_tet(g, P, level, coeff=g.make_coeff(*co), deg=2)
    A = orc.assemble(P, N, orc.Coeff(*co))
    L, D = orc.ilu0(A, N)
    ic = orc.interior_coords(N)
    got = np.array([t.exact_factor(*p) for p in ic])
    assert np.abs(got[:, :7] - L.T).max() < 1e-13
    assert np.abs(got[:, 7] - D).max() < 1e-13 * D.max()


@pytest.mark.parametrize("level,deg,kind", [(5, 4, "const"), (5, 6, "sinprod"), (6, 4, "sinprod")])
def test_surrogate_values_match_oracle_fit(g, orc, level, deg, kind):
    """The library's own fit (Householder QR of the ridge problem) and the
    oracle's (SVD least squares) give the same surrogate values."""
    N = 2 ** level
    P = si.macro_tet(33)
    co = ("sinprod", 1.0, 0.5, 0) if kind == "sinprod" else ("const", 1.0, 0.0, 0)
    t = host_tet(g, P, level, coeff=g.make_coeff(*co), deg=deg)
    pr = orc.Problem(P, level, orc.Coeff(*co), deg=deg)
    ic = orc.interior_coords(N)
    sel = np.arange(0, len(ic), max(1, len(ic) // 3000))
    got = np.array([t.eval_surrogate(*ic[i]) for i in sel])
    ref = np.vstack([pr.Ls[:, sel], pr.Dinv_s[sel]]).T
    err = np.abs(got - ref).max(0) / np.abs(ref).max(0)
    assert err.max() < 1e-8, err


def test_imported_surrogate_reproduces_oracle_values(g, orc):
    """Coefficients fitted by the oracle, imported into the library: the
    per-row tables evaluate to the oracle's direct tensor evaluation."""
    level, deg, N = 5, 6, 32
    P = si.macro_tet(34)
    pr = orc.Problem(P, level, orc.Coeff("sinprod", 1.0, 0.5), deg=deg)
    t = host_tet(g, P, level, coeff=g.make_coeff("sinprod", 1.0, 0.5), deg=deg)
    t.import_surrogate(pr.coefs)
    assert np.array_equal(t.export_surrogate(), pr.coefs.reshape(-1))
    ic = orc.interior_coords(N)
    got = np.array([t.eval_surrogate(*p) for p in ic])
    ref = np.vstack([pr.Ls, pr.Dinv_s]).T
    assert (np.abs(got - ref).max(0) / np.abs(ref).max(0)).max() < 1e-12


def test_invalid_inputs_raise(g):
    P = si.macro_tet(35)
    with pytest.raises(g.IluError) as e:
        host_tet(g, P, 1)
    assert e.value.status == g.ILU_EINVAL
    with pytest.raises(g.IluError):
        host_tet(g, P, 11)
    flat = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0.0]])
    with pytest.raises(g.IluError) as e:
        host_tet(g, flat, 3)
    assert "degenerate" in str(e.value)
    bad = P.copy(); bad[0, 0] = np.nan
    with pytest.raises(g.IluError):
        host_tet(g, bad, 3)
    with pytest.raises(g.IluError):
        host_tet(g, P, 3, coeff=g.make_coeff("const", -1.0))
    with pytest.raises(g.IluError):
        host_tet(g, P, 3, deg=13)
    t = host_tet(g, P, 3, deg=2)
    x = np.zeros(g.num_nodes(3)); b = np.zeros(g.num_nodes(3))
    with pytest.raises(g.IluError) as e:
        t.smooth_host(x, b, 1)
    assert e.value.status == g.ILU_ENODEV
    with pytest.raises(g.IluError):
        t.import_surrogate(np.zeros(5))
    with pytest.raises(g.IluError):
        t.eval_surrogate(0, 1, 1)


@pytest.mark.parametrize("level,kind", [(3, "const"), (4, "sinprod")])
def test_sgs_factors_match_oracle(g, orc, level, kind):
    """With ilu_opts.factor = SGS the library's exact factors are the
    symmetric Gauss-Seidel ones (a(p,p+d)/a(p+d,p+d) and a(p,p))."""
    N = 2 ** level
    P = si.macro_tet(34)
    co = ("sinprod", 1.0, 0.5, 0) if kind == "sinprod" else ("const", 1.0, 0.0, 0)
    t = host_tet(g, P, level, coeff=g.make_coeff(*co), deg=2, factor=g.FACTOR_SGS)
    A = orc.assemble(P, N, orc.Coeff(*co))
    L, D = orc.sgs_factors(A, N)
    got = np.array([t.exact_factor(*p) for p in orc.interior_coords(N)])
    assert np.abs(got[:, :7] - L.T).max() < 1e-13
    assert np.abs(got[:, 7] - D).max() < 1e-13 * D.max()


def test_sgs_surrogate_matches_oracle_fit(g, orc):
    level, deg, N = 5, 4, 32
    P = si.macro_tet(35)
    co = ("sinprod", 1.0, 0.5, 0)
    t = host_tet(g, P, level, coeff=g.make_coeff(*co), deg=deg, factor=g.FACTOR_SGS)
    pr = orc.Problem(P, level, orc.Coeff(*co), deg=deg, factor="sgs")
    Ls, Dinv = pr.surrogate_factors()
    ic = orc.interior_coords(N)
    got = np.array([t.eval_surrogate(*p) for p in ic[::5]])
    assert np.abs(got[:, :7] - Ls.T[::5]).max() < 1e-8
    assert np.abs(got[:, 7] - Dinv[::5]).max() < 1e-8 * np.abs(Dinv).max()


def test_v1_keeps_the_fit_and_runs_on_both_kernel_families(g):
    """Variant V1 stores boundary factors beside the same surrogate fit; it
    is accepted with either substitution kernel family."""
    P = si.macro_tet(33)
    a = g.Tet(P, 5, poly_degree=4, device=-1)
    b = g.Tet(P, 5, poly_degree=4, device=-1, boundary=g.BOUNDARY_V1)
    assert np.array_equal(a.export_surrogate(), b.export_surrogate())
    g.Tet(P, 5, poly_degree=4, device=-1, boundary=g.BOUNDARY_V1, kernel=g.KERNEL_BAND).close()
    with pytest.raises(g.IluError):
        g.Tet(P, 5, poly_degree=4, device=-1, boundary=5)


def test_tabulated_values_are_an_fp64_option(g):
    """ilu_opts.values: TABULATED needs F64 and level <= 9; unknown values
    are rejected before any device work."""
    P = si.macro_tet(36)
    g.Tet(P, 4, poly_degree=2, device=-1, precision=g.F64, values=g.VALUES_TABULATED).close()
    g.Tet(P, 4, poly_degree=2, device=-1, precision=g.MIXED, values=g.VALUES_ON_THE_FLY).close()
    for prec in [g.MIXED, g.F32]:
        with pytest.raises(g.IluError) as e:
            g.Tet(P, 4, poly_degree=2, device=-1, precision=prec, values=g.VALUES_TABULATED)
        assert e.value.status == g.ILU_EINVAL
    with pytest.raises(g.IluError) as e:
        g.Tet(P, 10, poly_degree=2, device=-1, precision=g.F64, values=g.VALUES_TABULATED)
    assert e.value.status == g.ILU_EINVAL
    with pytest.raises(g.IluError) as e:
        g.Tet(P, 4, poly_degree=2, device=-1, precision=g.F64, values=3)
    assert e.value.status == g.ILU_EINVAL


def test_handles_close_on_with_exit(g):
    P = si.macro_tet(37)
    with g.Tet(P, 3, poly_degree=2, device=-1) as t:
        assert t.h
        n = len(t.export_surrogate())
    assert t.h is None and n == 8 * 27
