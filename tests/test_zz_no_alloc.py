"""ilu_residual_noalloc: the residual entry point for callers that cannot let
the library allocate device memory (its scratch is a fixed array inside the
library).  Checked through the C ABI against ilu_residual on two calls in a
row; kept in a file of its own that pytest collects last."""
import ctypes

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


@pytest.mark.parametrize("prec,level,tol", [("MIXED", 6, 1e-13), ("F32", 5, 1e-6)])
def test_noalloc_residual_matches_ilu_residual(g, prec, level, tol):
    p = getattr(g, prec)
    dt = torch.float32 if p == g.F32 else torch.float64
    t = g.Tet(si.macro_tet(201), level, coeff=g.make_coeff("sinprod", 1.0, 0.5), poly_degree=4, precision=p)
    x = torch.tensor(si.boundary_data(level, 202), dtype=dt, device="cuda")
    b = torch.tensor(si.rhs(level, 203), dtype=dt, device="cuda")
    r_ref = torch.zeros_like(x)
    n_ref = t.residual(x, b, r_ref)
    L = g.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):  # the shared scratch keeps the previous call's contents
        r = torch.full_like(x, float("nan"))
        nd = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = L.ilu_residual_noalloc(t.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                    ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(nd.data_ptr()), stream)
        assert st == g.ILU_OK, L.ilu_last_error()
        torch.cuda.synchronize()
        got = r.cpu().numpy().astype(np.float64)
        ref = r_ref.cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
        assert abs(float(nd.item()) - n_ref) <= tol * n_ref


def test_noalloc_rejects_null_arguments(g):
    t = g.Tet(si.macro_tet(204), 4, poly_degree=2)
    x = torch.zeros(g.num_nodes(4), dtype=torch.float64, device="cuda")
    L = g.lib()
    st = L.ilu_residual_noalloc(t.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), None, None, None)
    assert st == g.ILU_EINVAL
