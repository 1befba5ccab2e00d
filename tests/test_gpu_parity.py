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


def gpu_tet(g, P, level, co, deg, prec, coefs, slabs=0, kernel=0):
    t = g.Tet(P, level, coeff=g.make_coeff(*co), poly_degree=deg if np.isscalar(deg) else 0,
              deg=deg, precision=prec, slabs=slabs, kernel=kernel)
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


@pytest.mark.parametrize("kernel", ["SLAB", "BAND", "PACKED"])
@pytest.mark.parametrize("prec", ["F32", "MIXED"])
@pytest.mark.parametrize("level,kind,deg", [(3, "const", 2), (4, "const", 4), (5, "sinprod", 6), (6, "const", 6),
                                            (6, "kappa_i", 3), (7, "sinprod", 6)])
def test_reduced_precision_per_sweep(g, orc, prec, level, kind, deg, kernel):
    """Each sweep, started from the oracle's current iterate, lands within
    1e-5 (relative) of the oracle's next iterate (every substitution kernel
    family)."""
    P, co, pr = problem(orc, level, 51 + level, kind, deg)
    N = 2 ** level
    p = getattr(g, prec)
    t = gpu_tet(g, P, level, co, deg, p, pr.coefs, kernel=getattr(g, "KERNEL_" + kernel))
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


@pytest.mark.parametrize("prec,kernel", [("F64", "SLAB"), ("MIXED", "SLAB"), ("MIXED", "BAND"), ("F32", "BAND")])
def test_slab_partition_is_bitwise_invariant(g, orc, prec, kernel):
    """The result does not depend on how the tet is split across CTAs (z-slabs
    of the slab kernels, layer stacks of the band kernels)."""
    level, deg = 6, 4
    P, co, pr = problem(orc, level, 61, "sinprod", deg)
    x0 = si.boundary_data(level, 62)
    b = si.rhs(level, 63)
    p = getattr(g, prec)
    dt = torch.float32 if p == g.F32 else torch.float64
    outs = []
    for slabs in [1, 2, 3, 7, 61]:
        t = gpu_tet(g, P, level, co, deg, p, pr.coefs, slabs=slabs, kernel=getattr(g, "KERNEL_" + kernel))
        xd = dev(x0, dt)
        t.smooth(xd, dev(b, dt), 2)
        outs.append(xd.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_band_kernels_at_full_bench_level(g, orc):
    """Level 9 (the size where the band kernels are chosen): four MIXED sweeps
    from x = 0 contract and stay finite, and the slab kernels give the same
    iterate to the FP32 bar.  The oracle check of the same sweeps is
    test_level9_sweep_solves_the_oracle_residual_equation."""
    level, deg = 9, 6
    P = si.macro_tet(5)
    t = g.Tet(P, level, coeff=g.make_coeff("const"), poly_degree=deg, precision=g.MIXED)
    assert t.N == 512
    b = dev(si.rhs(level, 6), torch.float64)
    x = torch.zeros_like(b)
    n0 = t.residual(x, b)
    norms = t.smooth(x, b, 4, norms=True)
    n4 = t.residual(x, b)
    # the smoother contracts on the level-9 problem and stays finite
    assert np.isfinite(norms).all() and abs(norms[0] - n0) <= 1e-9 * n0
    assert n4 < norms[-1] < norms[0]
    # the same sweeps with the slab kernels agree to the FP32 bar
    t2 = g.Tet(P, level, coeff=g.make_coeff("const"), poly_degree=deg, precision=g.MIXED, kernel=g.KERNEL_SLAB)
    x2 = torch.zeros_like(b)
    t2.smooth(x2, b, 4)
    assert rel(x.cpu().numpy(), x2.cpu().numpy()) < 1e-5


def level9_sample_points(N, seed, n_random=240):
    """Interior points for the level-9 checks: seeded random points plus
    points on each face of the interior, its edges and corners."""
    u = si.uniform(seed, 3 * n_random)
    pts = set()
    for k in range(n_random):
        z = 1 + int(u[3 * k + 2] * (N - 3))
        y = 1 + int(u[3 * k + 1] * (N - 2 - z))
        x = 1 + int(u[3 * k] * (N - 1 - y - z))
        pts.add((x, y, z))
    for m in (1, 2, 17, N // 3, N - 5):
        for a, c in ((1, m), (m, 1), (2, m)):
            pts.update({(1, a, c), (a, 1, c), (a, c, 1)})
            if a + c <= N - 2:
                pts.add((N - 1 - a - c, a, c))
    pts.update({(1, 1, 1), (N - 3, 1, 1), (1, N - 3, 1), (1, 1, N - 3)})
    return sorted(p for p in pts if p[0] >= 1 and p[1] >= 1 and p[2] >= 1 and sum(p) <= N - 1)


def sampled_sweep_check(g, orc, level, prec, kernel, tol, kind="const", deg=6, seed=5):
    """One sweep from x0 (Dirichlet data, interior 0) gives w = x1 - x0 =
    C~^-1 r.  At each sampled interior point the oracle evaluates the
    library's exported surrogate polynomials (direct tensor evaluation) on
    the point's neighbourhood and forms (L~ D~ L~^T w)_p, and computes r_p
    from its own element-assembled stencil; the two agree to `tol` relative
    to the largest |r_p|."""
    co = {"const": ("const", 1.0, 0.0, 0), "sinprod": ("sinprod", 1.0, 0.5, 0),
          "kappa_i": ("kappa_i", 0.0, 0.0, 2)}[kind]
    P = si.macro_tet(seed)
    p = getattr(g, prec)
    dt = torch.float32 if p == g.F32 else torch.float64
    t = g.Tet(P, level, coeff=g.make_coeff(*co), poly_degree=deg, precision=p,
              kernel=getattr(g, "KERNEL_" + kernel))
    N = t.N
    coefs = t.export_surrogate().reshape(8, -1)
    ids, _ = orc.interior_ids(N)
    npdt = np.float32 if p == g.F32 else np.float64
    x0 = si.boundary_data(level, 11).astype(npdt).astype(np.float64)
    x0[ids >= 0] = 0.0
    b = si.rhs(level, 12).astype(npdt).astype(np.float64)
    x = dev(x0, dt)
    t.smooth(x, dev(b, dt), 1)
    w = x.cpu().numpy().astype(np.float64) - x0
    del x
    t.close()
    at = lambda v: (lambda q: v[orc.index(N, *q)])
    oc = orc.Coeff(*co)
    cache = {}
    lhs, rhs = [], []
    for q in level9_sample_points(N, 13):
        lhs.append(orc.ldlt_apply_at(N, [deg] * 3, coefs, at(w), q, cache))
        rhs.append(orc.local_residual(P, N, oc, at(x0), at(b), q))
    lhs, rhs = np.array(lhs), np.array(rhs)
    assert len(rhs) > 250
    assert np.abs(lhs - rhs).max() <= tol * np.abs(rhs).max()


@pytest.mark.parametrize("prec,kernel,tol", [("MIXED", "BAND", 1e-5), ("F32", "BAND", 1e-5), ("MIXED", "SLAB", 1e-5),
                                             ("F64", "AUTO", 1e-12)])
def test_level9_sweep_solves_the_oracle_residual_equation(g, orc, prec, kernel, tol):
    """Level 9, the bench's single-tet size, element by element at sampled
    points (sampled_sweep_check)."""
    sampled_sweep_check(g, orc, 9, prec, kernel, tol)


@pytest.mark.parametrize("prec,kind", [("MIXED", "sinprod"), ("F32", "kappa_i"), ("F32", "const")])
def test_level8_packed_cluster_sweep_solves_the_oracle_residual_equation(g, orc, prec, kind):
    """Level 8, where the packed kernels run each tet on a cluster of two
    CTAs (rows of both CTAs read each other's rings), checked against the
    oracle at sampled points (sampled_sweep_check)."""
    sampled_sweep_check(g, orc, 8, prec, "PACKED", 1e-5, kind=kind, seed=7)


@pytest.mark.parametrize("boundary", ["V2", "V1"])
def test_level8_packed_cluster_sweeps_equal_slab_sweeps(g, boundary):
    """Level 8 on the whole grid: three MIXED sweeps of the two-CTA packed
    kernels land within 1e-5 of the slab kernels' sweeps (whose oracle parity
    is checked element by element at levels 2 to 7), for both boundary
    variants."""
    level, deg = 8, 5
    P = si.macro_tet(17)
    co = g.make_coeff("sinprod", 1.0, 0.5, 0)
    bnd = getattr(g, "BOUNDARY_" + boundary)
    x0 = si.boundary_data(level, 18)
    b = dev(si.rhs(level, 19), torch.float64)
    outs = []
    for kernel in (g.KERNEL_PACKED, g.KERNEL_SLAB):
        with g.Tet(P, level, coeff=co, poly_degree=deg, precision=g.MIXED, kernel=kernel, boundary=bnd) as t:
            x = dev(x0, torch.float64)
            t.smooth(x, b, 3)
            outs.append(x.cpu().numpy())
    assert np.isfinite(outs[0]).all()
    assert rel(outs[0], outs[1]) < 1e-5


@pytest.mark.parametrize("prec", ["F64", "MIXED", "F32"])
@pytest.mark.parametrize("level,kind", [(5, "sinprod"), (5, "const"), (6, "const"), (3, "const")])
def test_residual_matches_oracle(g, orc, prec, level, kind):
    """r = b - A x element by element: variable kappa (chunk form) and the
    constant stencil (strips of 30 points x 16 rows, several per layer at
    level 6, ragged at the layers' edges)."""
    P, co, pr = problem(orc, level, 71, kind, 3)
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


@pytest.mark.parametrize("prec,kernel", [("F64", "AUTO"), ("MIXED", "SLAB"), ("MIXED", "BAND"), ("F32", "BAND"),
                                         ("MIXED", "PACKED"), ("F32", "PACKED")])
def test_sgs_smoother_matches_oracle(g, orc, prec, kernel):
    """The symmetric Gauss-Seidel comparison smoother (ilu_opts.factor = SGS)
    runs through the same surrogate pipeline and kernels."""
    level, deg = 5, 4
    P = si.macro_tet(66)
    co = ("sinprod", 1.0, 0.5, 0)
    N = 2 ** level
    pr = orc.Problem(P, level, orc.Coeff(*co), deg=deg, factor="sgs")
    p = getattr(g, prec)
    t = g.Tet(P, level, coeff=g.make_coeff(*co), poly_degree=deg, precision=p,
              kernel=getattr(g, "KERNEL_" + kernel), factor=g.FACTOR_SGS)
    t.import_surrogate(pr.coefs)
    dt = torch.float32 if p == g.F32 else torch.float64
    x = si.boundary_data(level, 67)
    b = si.rhs(level, 68)
    Ls, Dinv = pr.surrogate_factors()
    xo = orc.smooth(pr.A, N, Ls, Dinv, x.copy(), b, 1)
    xd = dev(x, dt)
    t.smooth(xd, dev(b, dt), 1)
    tol = 1e-12 if p == g.F64 else 1e-5
    assert rel(xd.cpu().numpy().astype(np.float64), xo) < tol


@pytest.mark.parametrize("level,prec,kernel", [(4, "F64", 0), (6, "MIXED", 1), (6, "F32", 2), (5, "MIXED", 2)])
def test_stored_stencil_bitwise_equals_on_the_fly(g, orc, level, prec, kernel):
    """ilu_opts.stencil: in FP64 residuals (F64, MIXED) the stored
    coefficients are the on-the-fly FP64 sums applied in the same order, so
    sweeps and residuals agree bit for bit; F32 sweeps store and apply them in
    FP32.  All match the oracle."""
    P, co, pr = problem(orc, level, 70 + level, "sinprod", 4)
    p = getattr(g, prec)
    dt = torch.float32 if p == g.F32 else torch.float64
    x0 = si.boundary_data(level, 71)
    b = si.rhs(level, 72)
    out = []
    for stencil in [g.STENCIL_ON_THE_FLY, g.STENCIL_STORED]:
        t = g.Tet(P, level, coeff=g.make_coeff(*co), poly_degree=4, precision=p, kernel=kernel, stencil=stencil)
        t.import_surrogate(pr.coefs)
        xd, bd = dev(x0, dt), dev(b, dt)
        r = torch.zeros_like(bd)
        rn = t.residual(xd, bd, r)
        t.smooth(xd, bd, 2)
        out.append((xd.cpu().numpy(), r.cpu().numpy(), rn))
        t.close()
    if p == g.F32:
        assert rel(out[1][0], out[0][0]) < 1e-6 and rel(out[1][1], out[0][1]) < 1e-5
    else:
        assert np.array_equal(out[0][0], out[1][0])
        assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]
    Ls, Dinv = pr.surrogate_factors()
    xo = orc.smooth(pr.A, pr.N, Ls, Dinv, x0.copy(), b, 2)
    assert rel(out[1][0].astype(np.float64), xo) < (1e-12 if p == g.F64 else 2e-5)


@pytest.mark.parametrize("level,kind,deg,boundary,slabs", [
    (2, "const", 2, "V2", 0), (4, "const", 2, "V2", 0), (5, "sinprod", 6, "V2", 0), (6, "kappa_i", 9, "V2", 0),
    (5, "sinprod", 4, "V1", 0), (7, "sinprod", 6, "V2", 0), (7, "const", 3, "V2", 125), (6, "sinprod", 5, "V1", 7)])
def test_tabulated_values_bitwise_equal_on_the_fly(g, level, kind, deg, boundary, slabs):
    """ilu_opts.values: F64 substitutions that read the surrogate values from
    the set-up tables give the sweep of those that evaluate the row
    polynomials at every point, bit for bit (same FP64 Horner steps), for
    every padded row length (degrees 2, 6, 9), both boundary variants and
    several slab partitions; also after new coefficients are imported."""
    co = {"const": ("const", 1.0, 0.0, 0), "sinprod": ("sinprod", 1.0, 0.5, 0),
          "kappa_i": ("kappa_i", 0.0, 0.0, 2)}[kind]
    P = si.macro_tet(80 + level)
    bnd = g.BOUNDARY_V1 if boundary == "V1" else g.BOUNDARY_V2
    x0 = si.boundary_data(level, 81)
    b = si.rhs(level, 82)
    out = []
    for values in [g.VALUES_ON_THE_FLY, g.VALUES_TABULATED]:
        t = g.Tet(P, level, coeff=g.make_coeff(*co), poly_degree=deg, precision=g.F64, boundary=bnd,
                  slabs=slabs, values=values)
        xd, bd = dev(x0, torch.float64), dev(b, torch.float64)
        n1 = t.smooth(xd, bd, 2, norms=True)
        # re-import scaled coefficients: the tables must follow them
        c = t.export_surrogate()
        t.import_surrogate(c * (1.0 + 1e-3))
        n2 = t.smooth(xd, bd, 1, norms=True)
        out.append((xd.cpu().numpy(), n1, n2))
        t.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("level,kind,prec,kernel", [
    (3, "const", "F64", "SLAB"), (4, "sinprod", "F64", "SLAB"), (5, "kappa_i", "F64", "SLAB"),
    (6, "sinprod", "F64", "SLAB"), (5, "sinprod", "MIXED", "SLAB"), (7, "const", "MIXED", "SLAB"),
    (6, "kappa_i", "F32", "SLAB"), (5, "sinprod", "MIXED", "BAND"), (7, "const", "MIXED", "BAND"),
    (6, "kappa_i", "F32", "BAND"), (5, "sinprod", "MIXED", "PACKED"), (7, "const", "MIXED", "PACKED"),
    (6, "kappa_i", "F32", "PACKED")])
def test_v1_boundary_variant_matches_oracle(g, orc, level, kind, prec, kernel):
    """Variant V1: the stored exact factors (L^p_d and 1/D^p) at the
    cell-boundary points, surrogates elsewhere (the oracle's v1_factors)."""
    P, co, pr = problem(orc, level, 80 + level, kind, 4)
    p = getattr(g, prec)
    dt = torch.float32 if p == g.F32 else torch.float64
    t = g.Tet(P, level, coeff=g.make_coeff(*co), poly_degree=4, precision=p, boundary=g.BOUNDARY_V1,
              kernel=getattr(g, "KERNEL_" + kernel))
    t.import_surrogate(pr.coefs)
    x0 = si.boundary_data(level, 81)
    b = si.rhs(level, 82)
    Ls, Dinv = pr.surrogate_factors()
    L1, D1 = orc.v1_factors(pr.N, Ls, Dinv, pr.L, pr.D)
    xo = orc.smooth(pr.A, pr.N, L1, D1, x0.copy(), b, 2)
    xd = dev(x0, dt)
    t.smooth(xd, dev(b, dt), 2)
    assert rel(xd.cpu().numpy().astype(np.float64), xo) < (1e-12 if p == g.F64 else 2e-5)
    # and it differs from V2 where the surrogate misses the boundary factors
    # (at levels 3 and 4 every point is a sample and the fit is nearly exact)
    if level >= 5:
        x2 = orc.smooth(pr.A, pr.N, Ls, Dinv, x0.copy(), b, 2)
        assert rel(x2, xo) > 1e-9


def test_bench_configuration_matches_oracle(g, orc):
    """The default bench line's configuration exactly: the perturbed tet of
    seed 3, level 7, kappa = 1 + 0.5 sin sin sin, degree 6, MIXED, automatic
    kernel and stencil choices (slab kernels, stored stencils), b of seed 4,
    x0 = 0; two sweeps against the oracle."""
    level, deg = 7, 6
    P = si.macro_tet(3)
    co = ("sinprod", 1.0, 0.5, 0)
    pr = orc.Problem(P, level, orc.Coeff(*co), deg=deg)
    t = g.Tet(P, level, coeff=g.make_coeff(*co), poly_degree=deg, precision=g.MIXED)
    t.import_surrogate(pr.coefs)
    b = si.rhs(level, 4)
    x = np.zeros(si.num_nodes(level))
    Ls, Dinv = pr.surrogate_factors()
    xo = orc.smooth(pr.A, pr.N, Ls, Dinv, x.copy(), b, 2)
    xd = dev(x, torch.float64)
    t.smooth(xd, dev(b, torch.float64), 2)
    assert rel(xd.cpu().numpy(), xo) < 2e-5


@pytest.mark.parametrize("prec", ["F64", "F32"])
def test_exact_solution_is_a_fixed_point_at_level_9(g, prec):
    """At the level-9 size of the bench (where the oracle is too slow for a
    whole sweep): with b = A x* the sweep leaves x* in place, a property of
    x <- x + C~^-1 (b - A x) at any size (F64 slab kernels, F32 band kernels)."""
    level = 9
    p = getattr(g, prec)
    dt = torch.float32 if p == g.F32 else torch.float64
    t = g.Tet(si.macro_tet(5), level, coeff=g.make_coeff("const"), poly_degree=6, precision=p)
    xs = dev(si.interior_error(level, 7), dt)
    r = torch.zeros_like(xs)
    t.residual(xs, torch.zeros_like(xs), r)  # r = -A x* on the interior
    b = -r
    x = xs.clone()
    t.smooth(x, b, 1)
    d = (x - xs).abs().max().item() / xs.abs().max().item()
    assert d < (1e-12 if p == g.F64 else 1e-4), d
    # and from x = 0 the sweep moves towards x*
    x0 = torch.zeros_like(xs)
    t.smooth(x0, b, 2)
    assert (x0 - xs).norm().item() < (xs).norm().item()
