"""Host logic of the request loop without a GPU: argument checks, tickets,
waits with a time limit, statistics.  On a machine without a usable device
every admitted request ends with ILU_ENODEV instead of hanging."""
import numpy as np
import pytest

import seeded_inputs as si


@pytest.fixture(scope="module")
def g():
    import paper_2210_15280_gb300 as g
    g.build()
    return g


def test_create_rejects_bad_options(g):
    with pytest.raises(g.IluError) as e:
        g.Server(budget_bytes=1e9, device=-1)
    assert e.value.status == g.ILU_ENODEV
    with pytest.raises(g.IluError) as e:
        g.Server(budget_bytes=1e9, precision=7)
    assert e.value.status == g.ILU_EINVAL


def test_requests_without_device_fail_cleanly(g):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("this case needs a machine without a GPU")
    s = g.Server(budget_bytes=1e9, max_slots=2)
    b = si.rhs(3, 1)
    tks = [s.submit(si.macro_tet(1), 3, b, poly_degree=2) for _ in range(3)]
    assert len(set(tks)) == 3
    for tk in tks:
        r = s.wait(tk, timeout_ms=20000)
        assert r["status"] == g.ILU_ENODEV and r["x"] is None
    st = s.stats()
    assert st["submitted"] == 3 and st["failed"] == 3 and st["completed"] == 0
    with pytest.raises(g.IluError):
        s.wait(tks[0])  # released by the first wait
    with pytest.raises(ValueError):
        s.submit(si.macro_tet(1), 3, b[:-1])
    s.close()


def test_multigrid_request_checks(g):
    """Multigrid requests need level >= 3; methods beyond the four are
    rejected at submit; without a device they end with ILU_ENODEV."""
    torch = pytest.importorskip("torch")
    s = g.Server(budget_bytes=1e9, max_slots=1) if not torch.cuda.is_available() else None
    if s is None:
        pytest.skip("this case needs a machine without a GPU")
    with pytest.raises(g.IluError) as e:
        s.submit(si.macro_tet(1), 2, si.rhs(2, 1), method=g.MG_VCYCLE)
    assert e.value.status == g.ILU_EINVAL
    with pytest.raises(g.IluError) as e:
        s.submit(si.macro_tet(1), 3, si.rhs(3, 1), method=4)
    assert e.value.status == g.ILU_EINVAL
    tk = s.submit(si.macro_tet(1), 3, si.rhs(3, 1), method=g.MG_PCG, poly_degree=2)
    assert s.wait(tk, timeout_ms=20000)["status"] == g.ILU_ENODEV
    s.close()


def test_request_option_checks(g):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("this case needs a machine without a GPU")
    s = g.Server(budget_bytes=1e9, max_slots=1)
    for kw in [dict(orient=5), dict(boundary=3)]:
        with pytest.raises(g.IluError) as e:
            s.submit(si.macro_tet(1), 3, si.rhs(3, 1), **kw)
        assert e.value.status == g.ILU_EINVAL
    s.close()
