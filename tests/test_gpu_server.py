"""The request loop on the GPU: each result is the same alone and in a mix
of concurrently admitted requests, admission follows the memory budget, and
requests reach the solution of the assembled system."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import seeded_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

COEFFS = [("const", 1.0, 0.0, 0), ("sinprod", 1.0, 0.5, 0), ("kappa_i", 0.0, 0.0, 2)]


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_15280_gb300 as g
    g.build()
    return g


def requests(n, seed=6):
    mesh = si.macro_mesh(seed, n_tets=n)
    levels = si.batch_levels(seed + 1, n, 3, 5)
    out = []
    for i in range(n):
        L = int(levels[i])
        xb = np.zeros(si.num_nodes(L))
        out.append(dict(P=mesh[i], level=L, co=COEFFS[i % 3], deg=4 + i % 3, b=si.rhs(L, 700 + i),
                        x0=si.boundary_data(L, 800 + i) * 0.1, method=i % 2))
    return out


def submit(g, s, r):
    return s.submit(r["P"], r["level"], r["b"], coeff=g.make_coeff(*r["co"]), poly_degree=r["deg"],
                    method=r["method"], rtol=1e-8, max_iter=5000, x0=r["x0"])


@pytest.mark.parametrize("prec", ["MIXED", "F64"])
def test_same_result_alone_and_in_mix(g, orc, prec):
    reqs = requests(10)
    alone = []
    s1 = g.Server(max_slots=1, precision=getattr(g, prec))
    for r in reqs:
        alone.append(s1.wait(submit(g, s1, r)))
    s1.close()
    s8 = g.Server(max_slots=8, precision=getattr(g, prec))
    tks = [submit(g, s8, r) for r in reqs]
    mix = [s8.wait(tk) for tk in tks]
    st = s8.stats()
    s8.close()
    assert [a["status"] for a in alone] == [g.ILU_OK] * len(reqs)
    assert [m["status"] for m in mix] == [g.ILU_OK] * len(reqs)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["max_concurrent"] >= 2  # the requests overlapped
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    for i, (a, m) in enumerate(zip(alone, mix)):
        assert a["status"] == g.ILU_OK and m["status"] == g.ILU_OK, i
        assert a["rel_res"] <= 1e-8 and a["iters"] == m["iters"], i
        assert np.array_equal(a["x"], m["x"]), f"request {i} differs in the mix"
    # one of them against the assembled system's solution
    r, a = reqs[1], alone[1]
    N = 2 ** r["level"]
    pr = orc.Problem(r["P"], r["level"], orc.Coeff(*r["co"]), deg=r["deg"])
    S = orc.to_scipy(pr.A, N)
    ids, _ = orc.interior_ids(N)
    inn, bnd = np.nonzero(ids >= 0)[0], np.nonzero(ids < 0)[0]
    xs = r["x0"].copy()
    xs[inn] = spla.spsolve(S[inn][:, inn].tocsc(), r["b"][inn] - S[inn][:, bnd] @ r["x0"][bnd])
    assert np.abs(a["x"] - xs).max() < 1e-6 * np.abs(xs).max()
    assert np.array_equal(a["x"][bnd], r["x0"][bnd])


def test_admission_follows_memory_budget(g):
    reqs = requests(4, seed=12)
    for r in reqs:
        r["level"], r["b"], r["x0"] = 4, si.rhs(4, 1), np.zeros(si.num_nodes(4))
    # room for one request at a time (its tet and vectors), not two
    s = g.Server(budget_bytes=1.5e6, max_slots=4, precision=g.MIXED)
    tks = [submit(g, s, r) for r in reqs]
    res = [s.wait(tk) for tk in tks]
    st = s.stats()
    s.close()
    assert all(r["status"] == g.ILU_OK for r in res)
    assert st["max_concurrent"] == 1
    # a request that cannot fit at all fails, the loop goes on
    s = g.Server(budget_bytes=1e5, max_slots=2, precision=g.MIXED)
    r = s.wait(submit(g, s, reqs[0]))
    assert r["status"] == g.ILU_ENOMEM and r["x"] is None
    s.close()


def test_wait_with_time_limit_and_repeat_request(g):
    s = g.Server(max_slots=2, precision=g.MIXED)
    r = requests(1, seed=20)[0]
    r["level"], r["b"], r["x0"] = 6, si.rhs(6, 3), np.zeros(si.num_nodes(6))
    tk = submit(g, s, r)
    with pytest.raises(g.IluError) as e:
        s.wait(tk, timeout_ms=0, release=False)  # set-up alone takes longer
    assert e.value.status == g.ILU_ETIMEOUT
    first = s.wait(tk)
    second = s.wait(submit(g, s, r))  # same tet: resident, no set-up
    assert first["status"] == second["status"] == g.ILU_OK
    assert np.array_equal(first["x"], second["x"])
    assert second["latency_ms"] < first["latency_ms"]
    s.close()


def test_multigrid_requests(g, orc):
    """ILU_MG_VCYCLE / ILU_MG_PCG requests are served by resident multigrid
    hierarchies: a few cycles at any level, the same result alone and in a
    mix with single-level requests, and the assembled system's solution."""
    mesh = si.macro_mesh(9, n_tets=6)
    reqs = []
    for i in range(6):
        L = 4 + i % 3
        reqs.append(dict(P=mesh[i], level=L, co=COEFFS[i % 3], deg=5, b=si.rhs(L, 900 + i),
                         x0=si.boundary_data(L, 950 + i) * 0.1, method=[g.MG_VCYCLE, g.MG_PCG, g.PCG][i % 3]))
    s1 = g.Server(max_slots=1, precision=g.MIXED)
    alone = [s1.wait(submit(g, s1, r)) for r in reqs]
    s1.close()
    s4 = g.Server(max_slots=4, precision=g.MIXED)
    tks = [submit(g, s4, r) for r in reqs]
    mix = [s4.wait(tk) for tk in tks]
    s4.close()
    for i, (r, a, m) in enumerate(zip(reqs, alone, mix)):
        assert a["status"] == g.ILU_OK and m["status"] == g.ILU_OK, i
        assert a["rel_res"] <= 1e-8 and a["iters"] == m["iters"], i
        if r["method"] in (g.MG_VCYCLE, g.MG_PCG):
            assert a["iters"] <= 8, (i, a["iters"])
        assert np.array_equal(a["x"], m["x"]), i
    r, a = reqs[0], alone[0]
    N = 2 ** r["level"]
    pr = orc.Problem(r["P"], r["level"], orc.Coeff(*r["co"]))
    S = orc.to_scipy(pr.A, N)
    ids, _ = orc.interior_ids(N)
    inn, bnd = np.nonzero(ids >= 0)[0], np.nonzero(ids < 0)[0]
    xs = r["x0"].copy()
    xs[inn] = spla.spsolve(S[inn][:, inn].tocsc(), r["b"][inn] - S[inn][:, bnd] @ r["x0"][bnd])
    assert np.abs(a["x"] - xs).max() < 1e-6 * np.abs(xs).max()
    s = g.Server(max_slots=1, precision=g.MIXED)
    with pytest.raises(g.IluError):
        s.submit(mesh[0], 2, si.rhs(2, 1), method=g.MG_VCYCLE)
    s.close()


def test_requests_with_lfa_order_and_v1(g, orc):
    """A request may set the vertex order (LFA) and boundary variant of its
    set-up; its vectors then live in the layout of the reordered tet, and the
    result equals a standalone solve set up the same way."""
    P = np.array([[0, 0, 0.5], [0, 0, -0.5], [0.5, 10, 0], [-0.5, 10, 0]])
    perm = g.lfa_order(P)[0]
    assert perm != [0, 1, 2, 3]
    L = 5
    b = si.rhs(L, 990)
    s = g.Server(max_slots=2, precision=g.MIXED)
    tk = s.submit(P, L, b, poly_degree=5, method=g.MG_VCYCLE, rtol=1e-8, max_iter=50,
                  orient=g.ORIENT_LFA, boundary=g.BOUNDARY_V1)
    r = s.wait(tk)
    s.close()
    assert r["status"] == g.ILU_OK and r["rel_res"] <= 1e-8
    m = g.Multigrid(P, L, poly_degree=5, nu=3, precision=g.MIXED, orient=g.ORIENT_LFA, boundary=g.BOUNDARY_V1)
    x = torch.zeros(si.num_nodes(L), dtype=torch.float64, device="cuda")
    it, rel, ok = m.solve(x, torch.tensor(b, dtype=torch.float64, device="cuda"), g.RICHARDSON, 1e-8, 50)
    m.close()
    assert ok and it == r["iters"] and np.array_equal(x.cpu().numpy(), r["x"])
    # the solution of the reordered tet's assembled system
    Q = P[perm]
    N = 2 ** L
    S = orc.to_scipy(orc.assemble(Q, N), N)
    ids, _ = orc.interior_ids(N)
    inn = np.nonzero(ids >= 0)[0]
    xs = np.zeros_like(b)
    xs[inn] = spla.spsolve(S[inn][:, inn].tocsc(), b[inn])
    assert np.abs(r["x"] - xs).max() < 1e-6 * np.abs(xs).max()
