"""ilu_residual_noalloc: the residual entry point for callers that cannot let
the library allocate device memory (its scratch is a fixed array inside the
library).  Checked through the C ABI against ilu_residual on two calls in a
row; kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

import seeded_inputs as si

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_15280_gb300 as g
    g.build()
    return g


def test_noalloc_refuses_a_host_only_handle():
    """A handle set up without a device part (host-only set-up) is refused
    with ILU_ENODEV before anything is launched; this needs no GPU."""
    import paper_2210_15280_gb300 as g
    g.build()
    t = g.Tet(si.macro_tet(205), 4, poly_degree=2, device=-1)
    L = g.lib()
    fake = ctypes.c_void_p(16)  # never dereferenced: the handle is refused first
    st = L.ilu_residual_noalloc(t.h, fake, fake, fake, fake, None)
    assert st == g.ILU_ENODEV, L.ilu_last_error()
    t.close()


@pytest.mark.gpu
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


@pytest.mark.gpu
def test_noalloc_rejects_null_arguments(g):
    t = g.Tet(si.macro_tet(204), 4, poly_degree=2)
    x = torch.zeros(g.num_nodes(4), dtype=torch.float64, device="cuda")
    L = g.lib()
    st = L.ilu_residual_noalloc(t.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), None, None, None)
    assert st == g.ILU_EINVAL


@pytest.mark.gpu
def test_noalloc_refuses_a_failed_handle(g):
    """A handle whose bounded wait ran out (a wait limit of one poll) is
    refused with ILU_ECUDA, as by every other entry point."""
    level = 6
    b = torch.tensor(si.rhs(level, 207), dtype=torch.float64, device="cuda")
    L = g.lib()
    for attempt in range(5):  # a wait that never has to wait cannot run out
        t = g.Tet(si.macro_tet(206), level, poly_degree=4, precision=g.MIXED, max_wait_spins=1)
        x = torch.zeros_like(b)
        try:
            t.smooth(x, b, 2, norms=True)
        except g.IluError as e:
            assert e.status == g.ILU_ETIMEOUT, str(e)
            r = torch.zeros_like(b)
            nd = torch.zeros(1, dtype=torch.float64, device="cuda")
            st = L.ilu_residual_noalloc(t.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                        ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(nd.data_ptr()), None)
            assert st == g.ILU_ECUDA, L.ilu_last_error()
            t.close()
            return
        t.close()
    pytest.skip("no bounded wait ran out in five attempts")


@pytest.mark.gpu
def test_noalloc_leaves_the_current_device(g):
    """The call switches to the handle's device and back."""
    t = g.Tet(si.macro_tet(208), 5, poly_degree=2, precision=g.F64)
    x = torch.zeros(g.num_nodes(5), dtype=torch.float64, device="cuda")
    r = torch.zeros_like(x)
    nd = torch.zeros(1, dtype=torch.float64, device="cuda")
    before = torch.cuda.current_device()
    t.residual_noalloc(x, x, r, nd)
    torch.cuda.synchronize()
    assert torch.cuda.current_device() == before
    t.close()
