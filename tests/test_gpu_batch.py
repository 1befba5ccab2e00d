"""Batched smoothing (ilu_batch_*): tets of different levels, degrees and
coefficients in one batch give, tet by tet, the result of their own
single-tet sweeps (bit for bit: same kernels, same arithmetic), and the F64
batch matches the CPU oracle within 1e-12."""
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


COEFFS = [("const", 1.0, 0.0, 0), ("sinprod", 1.0, 0.5, 0), ("kappa_i", 0.0, 0.0, 2)]


def mixed_tets(g, prec, levels, degs, seed=6):
    """Tets of the jittered macro-mesh with the given levels and degrees,
    coefficients cycling through the three kinds."""
    mesh = si.macro_mesh(seed, n_tets=len(levels))
    out = []
    for i, (P, L, d) in enumerate(zip(mesh, levels, degs)):
        co = COEFFS[i % 3]
        out.append((P, L, d, co, g.Tet(P, L, coeff=g.make_coeff(*co), poly_degree=d, precision=prec)))
    return out


def vectors(tets, dtype, seed):
    xs, bs = [], []
    for i, (P, L, d, co, t) in enumerate(tets):
        n = si.num_nodes(L)
        xs.append(torch.tensor(si.boundary_data(L, seed + 2 * i), dtype=dtype, device="cuda"))
        bs.append(torch.tensor(si.rhs(L, seed + 2 * i + 1), dtype=dtype, device="cuda"))
        assert xs[-1].numel() == n
    return xs, bs


@pytest.mark.parametrize("prec", ["F64", "F32", "MIXED"])
def test_batch_equals_single_tet_sweeps(g, prec):
    # levels 3..7 (several groups), degrees across the register classes
    # (<= 3, 4..7) and, for F32, one above 7 (rows read from shared memory)
    levels = [6, 4, 7, 5, 4, 6, 3, 5]
    degs = [4, 2, 6, 5, 3, 9 if prec == "F32" else 4, 1, 6]
    tp = getattr(g, prec)
    dtype = torch.float32 if prec == "F32" else torch.float64
    tets = mixed_tets(g, tp, levels, degs)
    xs, bs = vectors(tets, dtype, 300)
    ref = [x.clone() for x in xs]
    for (P, L, d, co, t), x, b in zip(tets, ref, bs):
        t.smooth(x, b, 2)
    torch.cuda.synchronize()
    batch = g.Batch([t for *_, t in tets])
    batch.smooth(xs, bs, 2)
    for i, (x, r) in enumerate(zip(xs, ref)):
        assert torch.equal(x, r), f"tet {i} (level {levels[i]}, degree {degs[i]})"
    # replaying the captured graph, and re-capturing for another sweep count
    for (P, L, d, co, t), x, b in zip(tets, ref, bs):
        t.smooth(x, b, 3)
    batch.smooth(xs, bs, 1)
    batch.smooth(xs, bs, 2)
    for i, (x, r) in enumerate(zip(xs, ref)):
        assert torch.equal(x, r), f"tet {i} after replay"
    batch.close()


def test_f64_batch_matches_oracle(g, orc):
    levels, degs = [5, 3, 4], [4, 3, 5]
    tets = mixed_tets(g, g.F64, levels, degs, seed=9)
    prs = []
    for P, L, d, co, t in tets:
        pr = orc.Problem(P, L, orc.Coeff(*co), deg=d)
        t.import_surrogate(pr.coefs)
        prs.append(pr)
    xs, bs = vectors(tets, torch.float64, 400)
    x0 = [x.cpu().numpy().copy() for x in xs]
    batch = g.Batch([t for *_, t in tets])
    batch.smooth(xs, bs, 3)
    for (P, L, d, co, t), pr, x, xi, b in zip(tets, prs, xs, x0, bs):
        Ls, Dinv = pr.surrogate_factors()
        xo = xi.copy()
        orc.smooth(pr.A, 2 ** L, Ls, Dinv, xo, b.cpu().numpy(), 3)
        got = x.cpu().numpy()
        assert np.abs(got - xo).max() <= 1e-12 * np.abs(xo).max()


def test_batch_of_one_and_large_slab_request(g):
    tets = mixed_tets(g, g.MIXED, [6], [5])
    xs, bs = vectors(tets, torch.float64, 500)
    ref = [xs[0].clone()]
    tets[0][4].smooth(ref[0], bs[0], 2)
    b = g.Batch([tets[0][4]], slabs=61)  # one layer per slab
    b.smooth(xs, bs, 2)
    assert torch.equal(xs[0], ref[0])


def test_batch_rejects_bad_input(g):
    t64 = g.Tet(si.macro_tet(1), 4, poly_degree=3, precision=g.F64)
    t32 = g.Tet(si.macro_tet(2), 4, poly_degree=3, precision=g.F32)
    with pytest.raises(g.IluError):
        g.Batch([])
    with pytest.raises(g.IluError):
        g.Batch([t64, t32])  # mixed precisions
    b = g.Batch([t64])
    x = torch.zeros(si.num_nodes(4), dtype=torch.float64, device="cuda")
    with pytest.raises(g.IluError):
        b.smooth([x], [None], 1)
    b.smooth([x], [x.clone()], 0)  # no sweeps: nothing to do


def test_batch_with_v1_tets_equals_single_sweeps(g):
    """Tets set up with boundary variant V1 batch like any other (slab
    kernels; the boundary records travel in each tet's descriptor)."""
    mesh = si.macro_mesh(8, n_tets=4)
    tets = []
    for i, P in enumerate(mesh):
        co = COEFFS[i % 3]
        L = [5, 6, 5, 4][i]
        bnd = g.BOUNDARY_V1 if i % 2 == 0 else g.BOUNDARY_V2
        tets.append((P, L, 4, co, g.Tet(P, L, coeff=g.make_coeff(*co), poly_degree=4, precision=g.MIXED,
                                        boundary=bnd)))
    xs, bs = vectors(tets, torch.float64, 500)
    ref = [x.clone() for x in xs]
    for (P, L, d, co, t), x, b in zip(tets, ref, bs):
        t.smooth(x, b, 2)
    batch = g.Batch([t for *_, t in tets])
    batch.smooth(xs, bs, 2)
    for i, (x, r) in enumerate(zip(xs, ref)):
        assert torch.equal(x, r), i
    batch.close()


def test_f64_batch_mixing_tabulated_and_evaluated_tets(g):
    """F64 tets whose substitutions read tabulated values and tets that
    evaluate the polynomials run in separate groups of one batch; each gives
    its single-tet sweep bit for bit."""
    mesh = si.macro_mesh(12, n_tets=4)
    spec = [(5, 4, g.VALUES_TABULATED), (5, 4, g.VALUES_ON_THE_FLY), (6, 6, g.VALUES_AUTO), (4, 2, g.VALUES_ON_THE_FLY)]
    tets = []
    for i, (P, (L, d, v)) in enumerate(zip(mesh, spec)):
        co = COEFFS[i % 3]
        tets.append((P, L, d, co, g.Tet(P, L, coeff=g.make_coeff(*co), poly_degree=d, precision=g.F64, values=v)))
    xs, bs = vectors(tets, torch.float64, 500)
    ref = [x.clone() for x in xs]
    for (P, L, d, co, t), x, b in zip(tets, ref, bs):
        t.smooth(x, b, 2)
    torch.cuda.synchronize()
    batch = g.Batch([t for *_, t in tets])
    batch.smooth(xs, bs, 2)
    for i, (x, r) in enumerate(zip(xs, ref)):
        assert torch.equal(x, r), f"tet {i}"
    batch.close()
    for *_, t in tets:
        t.close()


@pytest.mark.parametrize("prec", ["F32", "MIXED"])
def test_batch_of_packed_tets_with_level8_clusters_equals_single_sweeps(g, prec):
    """Packed tets of levels 5 to 8 in one batch: the level-8 tets run on
    clusters of two CTAs, the others on one CTA each (groups by start
    quantum); every tet's sweeps equal its own handle's bit for bit."""
    levels, degs = [8, 7, 5, 8, 6], [6, 4, 3, 2, 5]
    mesh = si.macro_mesh(12, n_tets=len(levels))
    tp = getattr(g, prec)
    dtype = torch.float32 if prec == "F32" else torch.float64
    tets = []
    for i, (P, L, d) in enumerate(zip(mesh, levels, degs)):
        co = COEFFS[i % 3]
        tets.append((P, L, d, co, g.Tet(P, L, coeff=g.make_coeff(*co), poly_degree=d, precision=tp,
                                        kernel=g.KERNEL_PACKED)))
    xs, bs = vectors(tets, dtype, 700)
    ref = [x.clone() for x in xs]
    for (P, L, d, co, t), x, b in zip(tets, ref, bs):
        t.smooth(x, b, 2)
    batch = g.Batch([t for *_, t in tets])
    batch.smooth(xs, bs, 2)
    for i, (x, r) in enumerate(zip(xs, ref)):
        assert torch.isfinite(x).all()
        assert torch.equal(x, r), f"tet {i} (level {levels[i]}, degree {degs[i]})"
    batch.close()
    for *_, t in tets:
        t.close()
